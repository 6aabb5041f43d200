"""The paper's parallel test problems (Section 5) on the GPU: iteration counts
and attainable accuracy against the values the paper prints (needs a GB300).

The paper ran PETSc on 240 processes, whose reduction order differs from this
GPU's, so counts are compared with the paper's range and accuracy levels by
order of magnitude (tests/golden/ptp_reference.txt)."""
import os

import numpy as np
import pytest

from paper_1612_01395_gb300 import native, problems as P

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "ptp_reference.txt")


def golden():
    out = {}
    with open(GOLDEN) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                out[k] = float(v)
    return out


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    native.build()


def ptp(st):
    import torch
    s = native.Solver.from_stencil(st)
    b = s.spmv(torch.ones(st.n, dtype=torch.float64, device="cuda"))
    return s, b


def true_norm(s, b, x):
    return float((b - s.spmv(x)).norm())


@pytest.mark.parametrize("method,rp", [("standard", 0), ("pipelined", 0), ("pipelined", 100)],
                         ids=["bicgstab", "pbicgstab", "pbicgstab_rr"])
def test_ptp1_iterations_in_paper_range(method, rp):
    """PTP1 to 1e-6: 205 to 282 iterations over the paper's runs (Figure 3
    caption). The count depends on the reduction order (the paper's spans runs
    on 1 to 20 nodes), so 10 % is allowed on either side of that range."""
    g = golden()
    s, b = ptp(P.ptp1(1000))
    x, info = s.solve(b, rtol=1e-6, maxit=2000, method=method, replace_period=rp)
    assert info["status"] == native.PBCG_OK
    assert 0.9 * g["ptp1_iters_min"] <= info["iters"] <= 1.1 * g["ptp1_iters_max"], info["iters"]
    s.close()


def test_ptp1_attainable_accuracy_matches_paper():
    """Figure 4: BiCGStab 5.8e-12, p-BiCGStab 1.7e-9, p-BiCGStab-rr 2.5e-12
    within 2000 iterations (replacement every 100, at most 10).

    BiCGStab and p-BiCGStab-rr reach the attainable-accuracy floor, which is
    stable. p-BiCGStab without replacement stalls where the rounding errors of
    its recurrences have accumulated (Section 4.2), and where depends on the
    summation order. On this GPU, its best true residual over fixed runs of
    350..700 iterations is 7e-10 to 2e-8 over five block counts (the paper
    reports one run on 240 processes). So its pin is the median over those
    five summation orders, with the same factor 10, and it must stay two
    orders above the other two methods."""
    g = golden()
    s, b = ptp(P.ptp1(1000))
    x, _ = s.solve(b, rtol=1e-17, maxit=2000, method="standard")
    std = true_norm(s, b, x)
    x, _ = s.solve(b, rtol=1e-17, maxit=2000, replace_period=100, max_replacements=10)
    rr = true_norm(s, b, x)
    levels = []
    for grid in (304, 608, 760, 912, 1216):
        levels.append(min(true_norm(s, b, s.solve(b, rtol=0.0, maxit=k, fixed_iters=k, grid=grid)[0])
                          for k in range(350, 701, 25)))
    pipe = float(np.median(levels))
    for got, key in ((std, "ptp1_attained_bicgstab"), (rr, "ptp1_attained_pbicgstab_rr"),
                     (pipe, "ptp1_attained_pbicgstab")):
        assert g[key] / 10 <= got <= g[key] * 10, (key, got, levels)
    assert pipe > 100 * max(std, rr)
    s.close()


@pytest.mark.parametrize("method", ["standard", "pipelined"])
def test_ptp2_iterations_in_paper_range(method):
    """PTP2 to 1e-6: 1283 to 2112 iterations (Table 4), with the same 10 %
    allowance; the scaled tolerance corresponds to a true residual of at most
    3.0e-3."""
    g = golden()
    s, b = ptp(P.ptp2(1000))
    x, info = s.solve(b, rtol=1e-6, maxit=5000, method=method)
    assert info["status"] == native.PBCG_OK
    assert 0.9 * g["ptp2_iters_min"] <= info["iters"] <= 1.1 * g["ptp2_iters_max"], info["iters"]
    # a pipelined run's true residual trails its recursive one slightly
    assert true_norm(s, b, x) <= 1.5 * g["ptp2_true_residual_at_1e-6"]
    s.close()
