"""Why a float inner solve fails on the paper's transformer at 161x209 nodes,
checked with the oracle's matrices on the CPU (no library call).

The time levels' operator A = M + tau L (K_hat weights 29 on iron, 8e5 in
air, sigma 1e7 in the steel tank) has one isolated low-energy mode: after
symmetric diagonal scaling its smallest eigenvalue is about 2.5e-8 and the
next about 2e-4, so condition number x float rounding exceeds 1 for that mode
alone.  A float solve that acts on every mode (here a float32 sparse LU)
then returns the wrong amount of the mode, larger than the exact amount and
of the other sign, while staying accurate elsewhere; a correction that
overshoots in one mode makes the outer fixed point grow in it.  Deflating
the mode (its coefficient taken in double, the float solve on the rest)
restores the float solve's accuracy."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import workloads as W
from oracle import periodic as P


@pytest.fixture(scope="module")
def transformer():
    p = W.paper_transformer_problem(161, 209, 64)
    d = P.assemble(p)
    A = (d.M + d.tau * d.L).tocsc()
    Ds = sp.diags(1.0 / np.sqrt(A.diagonal()))
    As = (Ds @ A @ Ds).tocsc()
    vals, vecs = spla.eigsh(As, k=2, sigma=0, which="LM", tol=1e-10)
    order = np.argsort(vals)
    z = Ds @ vecs[:, order[0]]
    z /= np.sqrt(z @ (A @ z))   # unit in the energy norm
    return A, np.sort(vals), z


def test_one_isolated_low_mode(transformer):
    A, vals, _ = transformer
    assert vals[0] < 5e-8                 # condition number x float rounding > 1
    assert vals[1] / vals[0] > 1e3        # the rest is well separated
    assert vals[1] > 1e-4                 # condition number about 1e4 without it


def test_float_solve_overshoots_in_the_mode_and_deflation_fixes_it(transformer):
    A, _, z = transformer
    Az = A @ z
    lu32 = spla.splu(A.astype(np.float32).tocsc())
    rng = np.random.default_rng(0)
    b = rng.normal(size=A.shape[0])
    x = spla.spsolve(A, b)
    energy = lambda v: float(np.sqrt(v @ (A @ v)))
    c = z @ b                              # the mode's coefficient of the exact solution
    y = lu32.solve(b.astype(np.float32)).astype(np.float64)
    c_float = Az @ y
    assert abs(c_float - c) > abs(c)       # more than the whole exact amount wrong
    off = (y - x) - z * (Az @ (y - x))
    assert energy(off) < 1e-3 * energy(x)  # accurate off the mode
    # deflated: the mode in double, the float solve on the rest, its mode removed
    y1 = lu32.solve((b - Az * c).astype(np.float32)).astype(np.float64)
    xd = y1 - z * (Az @ y1) + z * c
    assert energy(xd - x) < 1e-4 * energy(x)
