"""The DFT-in-time exact periodic solve (Remark on parallel solvers,
Section 3) against the oracle: as the whole inner solve (time_levels = 1),
as the coarse solve of a truncated multigrid-in-time hierarchy, on
power-of-two step counts (shared-memory FFT) and others (direct transform),
on the nested grids (multigrid preconditioner) and on a generic mesh
(diagonal preconditioner).

Tolerances:
  * exact periodic solve in double (mode solves to 1e-12): 1e-10
  * converged fixed points: 1e-10 (FP64) and 1e-8 (mixed), as in the other
    parity tests
"""
import os

import numpy as np
import pytest

import workloads as W
from oracle import periodic as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
ptp = pytest.importorskip("paper_2502_21013_gb300.ptp")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def make_ctx(prob, structured=True, **opts):
    c = ptp.Context(0)
    ptp.load_problem(c, prob, structured=structured)
    o = ptp.default_opts(**opts)
    c.setup(o)
    return c, o


def cuda(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


DFT = dict(coarse_solver=1, time_levels=1, coarse_tol=1e-12, dft_max_it=80)


@pytest.mark.parametrize("N", [32, 24, 1, 2, 7])
def test_dft_periodic_solve_is_exact(N):
    """One application of the DFT solve is the exact periodic solve (nested
    grids: the mode solves are preconditioned by the tau L V-cycle)."""
    prob = W.unit_square_problem(33, N)
    d = P.assemble(prob)
    rng = np.random.default_rng(11)
    B = rng.normal(size=(d.n, d.N))
    ref = P.DFTSolver(d.M, d.L, d.tau, d.N).solve(B / d.tau)
    assert rel(ref, P.SpaceTimeLU(d.M, d.L, d.tau, d.N).solve(B / d.tau)) < 1e-12
    c, o = make_ctx(prob, precision=ptp.PTP_FP64, **DFT)
    X = torch.empty((d.n, d.N), dtype=torch.float64, device="cuda")
    r = c.periodic_solve_dev(cuda(B), X, 1, o)
    assert r < 1e-10
    assert rel(X.cpu().numpy(), ref) < 1e-10


def test_dft_periodic_solve_on_a_generic_mesh():
    """Unstructured Delaunay mesh: the mode solves are preconditioned by the
    diagonal of tau L and take more iterations, to the same exact result."""
    prob = W.delaunay_problem(120, 12, seed=3)
    d = P.assemble(prob)
    B = np.random.default_rng(14).normal(size=(d.n, d.N))
    ref = P.DFTSolver(d.M, d.L, d.tau, d.N).solve(B / d.tau)
    c, o = make_ctx(prob, False, precision=ptp.PTP_FP64, coarse_solver=1, time_levels=1, coarse_tol=1e-12,
                    dft_max_it=600)
    X = torch.empty((d.n, d.N), dtype=torch.float64, device="cuda")
    r = c.periodic_solve_dev(cuda(B), X, 1, o)
    assert r < 1e-10
    assert rel(X.cpu().numpy(), ref) < 1e-10


def test_dft_solve_in_mixed_mode_reads_and_writes_float_levels():
    """Mixed precision: the level right-hand side and correction are float,
    the transform and mode solves double, so one solve is exact up to the
    float rounding of its input and output, whatever the scale of B."""
    prob = W.config_plain_fp64()
    d = P.assemble(prob)
    B = np.random.default_rng(12).normal(size=(d.n, d.N))
    ref = P.DFTSolver(d.M, d.L, d.tau, d.N).solve(B / d.tau)
    c, o = make_ctx(prob, precision=ptp.PTP_MIXED, **DFT)
    X = torch.empty((d.n, d.N), dtype=torch.float64, device="cuda")
    for scale in (1.0, 1e-12):
        r = c.periodic_solve_dev(cuda(B * scale), X, 1, o)
        assert r < 1e-6
        assert rel(X.cpu().numpy() / scale, ref) < 1e-5


@pytest.mark.parametrize("levels", [2, 3])
def test_dft_coarse_level_of_a_truncated_hierarchy(levels):
    """V-cycles whose last level (N / 2^(levels-1) steps) is solved by the DFT
    converge to the exact periodic solve."""
    prob = W.config_plain_fp64()
    d = P.assemble(prob)
    B = np.random.default_rng(13).normal(size=(d.n, d.N))
    ref = P.DFTSolver(d.M, d.L, d.tau, d.N).solve(B / d.tau)
    c, o = make_ctx(prob, precision=ptp.PTP_FP64, coarse_solver=1, time_levels=levels, coarse_tol=1e-12,
                    dft_max_it=80)
    X = torch.empty((d.n, d.N), dtype=torch.float64, device="cuda")
    r1 = c.periodic_solve_dev(cuda(B), X, 1, o)
    assert r1 < 0.5
    r = c.periodic_solve_dev(cuda(B), X, 40, o)
    assert r < 1e-10
    assert rel(X.cpu().numpy(), ref) < 1e-9


@pytest.mark.parametrize("precision,tol,bar", [("fp64", 1e-13, 1e-10), ("mixed", 1e-11, 1e-8)])
@pytest.mark.parametrize("levels", [1, 2])
def test_fixed_point_with_dft_inner_solve_against_stored_oracle(precision, tol, bar, levels):
    """The whole nonlinear solve with the DFT as inner solver (levels = 1) and
    as the coarse solve of the two-level method (levels = 2) reaches the
    oracle's fixed point."""
    prob = W.config_plain_fp64()
    Uo = np.load(os.path.join(GOLDEN, "square33_N32_oracle.npz"))["U"]
    prec = ptp.PTP_FP64 if precision == "fp64" else ptp.PTP_MIXED
    c, o = make_ctx(prob, precision=prec, tol=tol, max_outer=20000, coarse_solver=1, time_levels=levels,
                    coarse_tol=1e-10, dft_max_it=40)
    U, st, rc = c.solve(o)
    assert rc == ptp.PTP_OK and st.converged
    assert st.time_levels == levels
    assert rel(U, Uo) < bar


def test_dft_bottom_of_a_hierarchy_that_ends_on_an_odd_step_count():
    """N = 24 coarsens 24 -> 12 -> 6 -> 3; the 3-step bottom has no sum /
    difference split, and the DFT solve (direct transform) closes it."""
    prob = W.unit_square_problem(17, 24)
    d = P.assemble(prob)
    ref = P.fixed_point(prob, d, tol=1e-13, max_it=50000)
    assert ref.converged
    c, o = make_ctx(prob, precision=ptp.PTP_FP64, tol=1e-13, max_outer=20000, coarse_solver=1, coarse_tol=1e-10)
    U, st, rc = c.solve(o)
    assert rc == ptp.PTP_OK and st.time_levels == 4
    assert rel(U, ref.U) < 1e-10
    cv, ov = make_ctx(prob, precision=ptp.PTP_FP64, tol=1e-13, max_outer=10)
    with pytest.raises(ptp.PtpError):   # without the DFT the 3-step bottom has no exact solve
        cv.solve(ov)


def test_dft_solver_rejects_levels_beyond_its_limit():
    prob = W.unit_square_problem(5, 1024)
    c = ptp.Context(0)
    ptp.load_problem(c, prob)
    with pytest.raises(ptp.PtpError):
        c.setup(ptp.default_opts(coarse_solver=1, time_levels=1))
