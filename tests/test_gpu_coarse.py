"""The coarsest time level's solve tau_c L x = b.

On a uniform structured grid with K_hat = nu_max A and (nx - 1), (ny - 1)
powers of two the library solves it directly by sine transforms along the
rows and the columns (exact up to rounding); otherwise by PCG to coarse_tol.
With one time step (N = 1) the periodic system of Problem 1 is exactly that
solve, so the library's periodic solve is checked against a sparse direct
solve of the oracle's tau L."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as W
from oracle import periodic as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
ptp = pytest.importorskip("paper_2502_21013_gb300.ptp")


def _ctx(prob, **kw):
    c = ptp.Context(0)
    ptp.load_problem(c, prob)
    o = ptp.default_opts(**kw)
    c.setup(o)
    return c, o


CASES = [
    ("square33", lambda: W.unit_square_problem(33, 1)),
    ("square257", lambda: W.unit_square_problem(257, 1)),
    ("rectangle65x33", lambda: W.transformer_problem(65, 33, 1)),      # hx = hy on [0,2]x[0,1]
    ("rectangle33x33", lambda: W.transformer_problem(33, 33, 1)),      # hx = 2 hy
]


@pytest.mark.parametrize("name,make", CASES, ids=[c[0] for c in CASES])
def test_direct_coarse_solve_is_exact(name, make):
    prob = make()
    d = P.assemble(prob)
    rng = np.random.default_rng(8)
    b = rng.normal(size=(d.n, 1))
    x_ref = spla.spsolve((d.tau * d.L).tocsc(), b[:, 0])
    c, o = _ctx(prob, precision=ptp.PTP_FP64, coarse_direct=1)
    B = torch.tensor(b, device="cuda")
    X = torch.empty_like(B)
    rel = c.periodic_solve_dev(B, X, 1, o)
    x = X.cpu().numpy()[:, 0]
    assert np.linalg.norm(x - x_ref) <= 1e-12 * np.linalg.norm(x_ref)
    assert rel <= 1e-13
    # the iterative coarse solve stops at coarse_tol (1e-6) after at most coarse_max_it steps
    c2, o2 = _ctx(prob, precision=ptp.PTP_FP64, coarse_direct=0)
    X2 = torch.empty_like(B)
    rel2 = c2.periodic_solve_dev(B, X2, 1, o2)
    assert rel2 > rel


def test_direct_coarse_solve_in_the_fixed_point():
    """Fixed points with the direct and the iterative coarsest solve both
    reach the stored oracle solution (33x33, N = 32)."""
    import os
    prob = W.unit_square_problem(33, 32)
    Uo = np.load(os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "square33_N32_oracle.npz"))["U"]
    for direct in (1, 0):
        for precision, tol, bar in ((ptp.PTP_FP64, 1e-13, 1e-10), (ptp.PTP_MIXED, 1e-11, 1e-8)):
            c, o = _ctx(prob, precision=precision, tol=tol, max_outer=20000, coarse_direct=direct)
            U, st, rc = c.solve(o)
            assert rc == ptp.PTP_OK
            assert np.linalg.norm(U - Uo) / np.linalg.norm(Uo) < bar, (direct, precision)


def test_direct_coarse_solve_not_taken_off_its_grids():
    """K_hat weights (the paper's transformer) or a generic mesh: the
    iterative coarse solve is used and the solves still work."""
    prob = W.unit_square_problem(17, 1)
    d = P.assemble(prob)
    b = np.random.default_rng(2).normal(size=(d.n, 1))
    c, o = _ctx(prob.replace(khat_e=np.full(prob.n_tri, prob.nu_max)), precision=ptp.PTP_FP64, coarse_direct=1,
                coarse_tol=1e-12, coarse_max_it=200)
    B = torch.tensor(b, device="cuda")
    X = torch.empty_like(B)
    rel = c.periodic_solve_dev(B, X, 1, o)
    assert rel <= 1e-11
