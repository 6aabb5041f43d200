"""The batched benchmark's flop count (host logic, no GPU): per system, the
SpMVs of the setup, the iterations, the replacements and the final true
residual at 2 flops per stored entry, plus Algorithm 9's 42 flops per row and
iteration."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_batched_flops_counts_each_system():
    # system 0: 3 rows, 7 entries, 2 iterations, no replacement:
    #   SpMVs 3 + 4 = 7 -> 7 * 2 * 7 = 98; rows 2 * 42 * 3 = 252
    # system 1: 5 rows, 13 entries, 4 iterations, 1 replacement:
    #   SpMVs 3 + 8 + 3 = 14 -> 14 * 2 * 13 = 364; rows 4 * 42 * 5 = 840
    assert bench.batched_flops([3, 5], [7, 13], [2, 4], [0, 1]) == 98 + 252 + 364 + 840


def test_batched_flops_of_an_unconverged_empty_batch():
    assert bench.batched_flops([], [], [], []) == 0.0
    # a system stopped before its first iteration still pays setup and residual
    assert bench.batched_flops(np.array([4]), np.array([10]), np.array([0]), np.array([0])) == 3 * 2 * 10
