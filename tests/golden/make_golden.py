"""Writes the stored expected values used by the GPU parity tests.

Every value here is computed by the CPU oracle alone (package `oracle`),
never by the CUDA library.  Run from the repository root:
    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402
from oracle import periodic as P  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    # The 33x33, N = 32 unit-square workload (2048 triangles, J0 = 50),
    # solved by the fixed point of eq. (iter1)-(iter2) with exact DFT inner
    # solves to a relative residual of 1e-13.
    prob = W.config_plain_fp64()
    d = P.assemble(prob)
    res = P.fixed_point(prob, d, tol=1e-13, max_it=20000)
    assert res.converged
    np.savez_compressed(os.path.join(HERE, "square33_N32_oracle.npz"), U=res.U,
                        iterations=res.iterations, res_history=np.array(res.res_history))
    print("square33_N32: iterations", res.iterations, "final rel. residual",
          res.res_history[-1] / res.res_history[0])


if __name__ == "__main__":
    main()
