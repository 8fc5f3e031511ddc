"""The static initialisation of Section 4 on the GPU against the oracle.

With sigma = 0 the time steps decouple into K(u^n) = f^n; the library solves
all N of them at once by eq. (iter1) with M = 0 and batched multigrid PCG.
Tolerances as in the other parity tests: 1e-10 (FP64, both sides solved to
1e-13) and 1e-8 (mixed, solved to 1e-11).
"""
import numpy as np
import pytest

import workloads as W
from oracle import periodic as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
ptp = pytest.importorskip("paper_2502_21013_gb300.ptp")


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def make_ctx(prob, structured=True, **opts):
    c = ptp.Context(0)
    ptp.load_problem(c, prob, structured=structured)
    o = ptp.default_opts(**opts)
    c.setup(o)
    return c, o


CASES = {
    "square33_N32": lambda: W.config_plain_fp64(),
    "square17_N8_saturated": lambda: W.unit_square_problem(17, 8, amps=(4000.0,)),
    "transformer33x17_N6": lambda: W.transformer_problem(33, 17, 6),
}


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision,tol,bar", [("fp64", 1e-13, 1e-10), ("mixed", 1e-11, 1e-8)])
def test_static_solve_against_oracle(name, precision, tol, bar):
    prob = CASES[name]()
    d = P.assemble(prob)
    Uo, r = P.static_solve(prob, d)
    assert r < 1e-13
    prec = ptp.PTP_FP64 if precision == "fp64" else ptp.PTP_MIXED
    c, o = make_ctx(prob, precision=prec, tol=tol, max_outer=20000)
    U, st, rc = c.static_solve(o)
    assert rc == ptp.PTP_OK and st.converged and st.outer_iterations > 0
    assert rel(U, Uo) < bar
    F = P.source(prob, d)
    assert np.linalg.norm(F - P.K_free(prob, d, U)) <= 1.01 * tol * np.linalg.norm(F)
    # the device-pointer form gives the same iterate
    Ud = torch.empty((d.n, d.N), dtype=torch.float64, device="cuda")
    st2, rc2 = c.static_solve_dev(Ud, o)
    assert rc2 == ptp.PTP_OK and st2.outer_iterations == st.outer_iterations
    assert np.array_equal(Ud.cpu().numpy(), U)


def test_static_solve_on_a_generic_mesh():
    prob = W.delaunay_problem(200, 6, seed=2, amp=2000.0)
    d = P.assemble(prob)
    Uo, _ = P.static_solve(prob, d)
    c, o = make_ctx(prob, False, precision=ptp.PTP_FP64, tol=1e-13, max_outer=20000)
    U, st, rc = c.static_solve(o)
    assert rc == ptp.PTP_OK
    assert rel(U, Uo) < 1e-10


@pytest.mark.parametrize("precision,tol,bar", [("fp64", 1e-13, 1e-10), ("mixed", 1e-11, 1e-8)])
def test_periodic_solve_started_from_the_static_solutions(precision, tol, bar):
    """init_static: the solve first reaches the static solutions, then runs
    the periodic iteration from them; the limit is the oracle's periodic
    solution, and the periodic residual at the start is the one of the static
    solutions, F - A(U_static) = -M d_tau U_static."""
    prob = W.unit_square_problem(17, 16, amps=(2000.0,))
    d = P.assemble(prob)
    ref = P.fixed_point(prob, d, tol=1e-13, max_it=50000)
    assert ref.converged
    Us, _ = P.static_solve(prob, d)
    prec = ptp.PTP_FP64 if precision == "fp64" else ptp.PTP_MIXED
    c, o = make_ctx(prob, precision=prec, tol=max(tol, 1e-12), max_outer=20000, init_static=1, init_tol=1e-11)
    U, st, rc = c.solve(o)
    assert rc == ptp.PTP_OK and st.converged
    assert st.init_iterations > 0 and st.init_ms > 0
    assert rel(U, ref.U) < bar
    r_static = np.linalg.norm(P.residual(prob, d, Us))
    assert abs(st.res0 - r_static) <= 1e-6 * r_static
    assert st.res0 < np.linalg.norm(P.source(prob, d))


def test_zero_conductivity_periodic_solve_equals_static_solve():
    """sigma = 0: the periodic problem is the static one, for the GPU too."""
    prob = W.unit_square_problem(17, 8, amps=(3000.0,))
    prob = prob.replace(sigma_e=np.zeros(prob.n_tri))
    c, o = make_ctx(prob, precision=ptp.PTP_FP64, tol=1e-13, max_outer=20000)
    Us, st, rc = c.static_solve(o)
    assert rc == ptp.PTP_OK
    Up, st2, rc2 = c.solve(o)
    assert rc2 == ptp.PTP_OK
    assert rel(Up, Us) < 1e-10
