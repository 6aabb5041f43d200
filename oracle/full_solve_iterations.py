"""Run the oracle to convergence on the 256^3 convection-diffusion system and
print its iteration counts (test infrastructure; slow: tens of minutes on one
core). The benchmark's CPU-baseline leg times a bounded sample of oracle
iterations and scales it by these counts.

    python -m oracle.full_solve_iterations [n]
"""
import sys
import time

import numpy as np

import oracle
from paper_1612_01395_gb300 import problems as P


def main(n=256):
    st = P.cd3d_trig(n)
    A = P.stencil_to_csr(st)
    b = oracle.spmv(A, P.splitmix64_uniform(0, A.n))
    for name, fn, kw in [("pbicgstab_rr50", oracle.pbicgstab, dict(replace_period=50)),
                         ("bicgstab", oracle.bicgstab, {})]:
        t0 = time.time()
        r = fn(A, b, rtol=1e-8, maxit=20000, **kw)
        print(f"{name} n={n}^3 iters={r.iters} status={r.status} rel_res_true={r.rel_res_true:.3e} "
              f"seconds={time.time() - t0:.1f}", flush=True)


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 256)
