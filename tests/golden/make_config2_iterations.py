"""Writes config2_sync_fp64_cg20_iterations.txt by running the CPU oracle.

Workload: 2D Poisson 1024 x 1024, b uniform in [-1, 1] (SplitMix64 seed 1),
regular 16 x 16 partition, overlap 4, local CG with 20 steps in FP64,
synchronous RAS from x0 = 0 to relative residual 1e-8. Calls only oracle/
(and the shared input generators). Run: python tests/golden/make_config2_iterations.py
"""
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import problems  # noqa: E402


def main():
    N, px, gamma, m, tol = 1024, 16, 4, 20, 1e-8
    A = problems.poisson2d(N)
    b = problems.rhs_uniform(A.n, 1)
    part = oracle.partition_regular2d(N, N, px, px)
    t0 = time.time()
    _, it, hist = oracle.ras_sync(A, b, part, px * px, gamma, oracle.CG, oracle.FP64, m, tol=tol,
                                  max_iter=200000, nthreads=os.cpu_count())
    out = os.path.join(HERE, "config2_sync_fp64_cg20_iterations.txt")
    with open(out, "w") as f:
        f.write("# Synchronous RAS iterations of the CPU oracle to relative residual 1e-8:\n")
        f.write("# 2D Poisson 1024^2, uniform b (seed 1), regular 16x16, overlap 4, local CG-20 FP64.\n")
        f.write(f"# written by tests/golden/make_config2_iterations.py ({time.time() - t0:.0f} s,"
                f" final relres {hist[-1]:.3e})\n")
        f.write(f"{it}\n")
    print(it, hist[-1])


if __name__ == "__main__":
    main()
