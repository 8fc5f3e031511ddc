"""Parity of the CUDA path (through the C ABI) against the CPU oracle.

Tolerances (relative Euclidean norms over the whole space-time block):
  * operator applications in double: 1e-13 (only the summation order differs)
  * operator applications in float:  1e-6  (float rounding of values and data)
  * converged solutions, FP64 path:  1e-10 (both sides solved to 1e-13)
  * converged solutions, mixed path: 1e-8  (GPU solved to 1e-11 with the
    double outer residual)
"""
import math
import os

import numpy as np
import pytest
import scipy.sparse.linalg as spla

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


def cuda(a, dtype=torch.float64):
    return torch.tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


PROBLEMS = {
    "square33_N32": lambda: W.config_plain_fp64(),
    "transformer33x17_N8": lambda: W.transformer_problem(33, 17, 8),
    "square9_N4_strong": lambda: W.unit_square_problem(9, 4, amps=(3000.0,)),
    "square17_N6": lambda: W.unit_square_problem(17, 6),
    # structured grids whose N is a multiple of 16 take the fused one-pass K1
    # (time tiles of 16 columns): three tiles, a rectangle, saturated iron
    "square33_N48_strong": lambda: W.unit_square_problem(33, 48, amps=(500.0,)),
    "transformer65x33_N16": lambda: W.transformer_problem(65, 33, 16),
}


# ---------------------------------------------------------------------------
# a1 / a2: source and outer residual (K1)
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("name", list(PROBLEMS))
@pytest.mark.parametrize("structured,k1_fused", [(True, 0), (True, 1), (False, 0)])
def test_source_and_residual(name, structured, k1_fused):
    """k1_fused = 1 takes the one-pass structured kernel where N is a multiple
    of 16 (the others fall back to the element and node passes)."""
    prob = PROBLEMS[name]()
    d = P.assemble(prob)
    c, _ = make_ctx(prob, structured, precision=ptp.PTP_FP64, k1_fused=k1_fused)
    F = c.source()
    assert rel(F, P.source(prob, d)) < 1e-14
    rng = np.random.default_rng(1)
    for scale in (1e-3, 1.0):   # linear and strongly saturated iron
        U = rng.normal(scale=scale, size=(d.n, d.N))
        R, nrm = c.residual(U)
        Ro = P.residual(prob, d, U)
        assert rel(R, Ro) < 1e-13
        assert abs(nrm - np.linalg.norm(Ro)) <= 1e-13 * np.linalg.norm(Ro)


def test_residual_device_pointers_and_zero_state():
    prob = W.config_plain_fp64()
    d = P.assemble(prob)
    c, _ = make_ctx(prob, precision=ptp.PTP_FP64)
    U = torch.zeros((d.n, d.N), dtype=torch.float64, device="cuda")
    R = torch.empty_like(U)
    nrm = c.residual_dev(U, R)
    F = P.source(prob, d)
    assert rel(R.cpu().numpy(), F) < 1e-15            # R(0) = F
    assert abs(nrm - np.linalg.norm(F)) < 1e-13 * np.linalg.norm(F)


# ---------------------------------------------------------------------------
# a5 / a6: SpMM with N right-hand sides, periodic operator, batched PCG
# ---------------------------------------------------------------------------

def _levels(c):
    return c.sizes()[3]


def test_shifted_and_periodic_operators_every_level():
    prob = W.config_plain_fp64()
    d = P.assemble(prob)
    c, _ = make_ctx(prob, precision=ptp.PTP_FP64)
    rng = np.random.default_rng(2)
    for lev in range(_levels(c)):
        Nl = d.N >> lev
        tau = prob.T / Nl
        X = rng.normal(size=(d.n, Nl))
        Y = torch.empty((d.n, Nl), dtype=torch.float64, device="cuda")
        c.apply_shifted_dev(lev, cuda(X), Y)
        ref = (d.M + tau * d.L) @ X
        assert rel(Y.cpu().numpy(), ref) < 1e-14
        Yf = torch.empty((d.n, Nl), dtype=torch.float32, device="cuda")
        c.apply_shifted_dev(lev, cuda(X, torch.float32), Yf)
        assert rel(Yf.double().cpu().numpy(), ref) < 1e-6
        c.periodic_apply_dev(lev, cuda(X), Y)
        refp = tau * (P.periodic_matrix(d.M, d.L, tau, Nl) @ X.ravel()).reshape(X.shape)
        assert rel(Y.cpu().numpy(), refp) < 1e-13


@pytest.mark.parametrize("prec", ["jacobi", "gmg"])
def test_batched_pcg(prec):
    prob = W.config_plain_fp64()
    d = P.assemble(prob)
    sp = ptp.PTP_PREC_JACOBI if prec == "jacobi" else ptp.PTP_PREC_GMG
    c, _ = make_ctx(prob, precision=ptp.PTP_FP64, spatial_prec=sp)
    rng = np.random.default_rng(3)
    for lev in (0, _levels(c) - 2):
        Nl = d.N >> lev
        tau = prob.T / Nl
        B = rng.normal(size=(d.n, Nl))
        B[:, 0] = 0.0   # a zero column must stay zero (no NaN from 0/0)
        ref = spla.spsolve((d.M + tau * d.L).tocsc(), B)
        X = torch.empty((d.n, Nl), dtype=torch.float64, device="cuda")
        it = c.spatial_solve_dev(lev, cuda(B), X, 1e-12, 2000)
        assert it < (30 if prec == "gmg" else 2000)
        assert rel(X.cpu().numpy(), ref) < 1e-9
        Xf = torch.empty((d.n, Nl), dtype=torch.float32, device="cuda")
        c.spatial_solve_dev(lev, cuda(B, torch.float32), Xf, 1e-6, 2000)
        assert rel(Xf.double().cpu().numpy(), ref) < 1e-4
        assert torch.isfinite(Xf).all()


# ---------------------------------------------------------------------------
# a4 / a5 / a7: multigrid in time for the periodic linear system
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("coarse_steps", [1, 2])
def test_multigrid_in_time_converges_to_exact_periodic_solve(coarse_steps):
    prob = W.config_plain_fp64()
    d = P.assemble(prob)
    rng = np.random.default_rng(4)
    B = rng.normal(size=(d.n, d.N))
    # the exact solution of (M + tau L) x^n - M x^{n-1} = b^n, x^0 = x^N
    ref = P.DFTSolver(d.M, d.L, d.tau, d.N).solve(B / d.tau)
    c, o = make_ctx(prob, precision=ptp.PTP_FP64, coarse_steps=coarse_steps, coarse_tol=1e-12,
                    coarse_max_it=40)
    X = torch.empty((d.n, d.N), dtype=torch.float64, device="cuda")
    r1 = c.periodic_solve_dev(cuda(B), X, 1, o)
    assert r1 < 0.5
    r = c.periodic_solve_dev(cuda(B), X, 40, o)
    assert r < 1e-10
    assert rel(X.cpu().numpy(), ref) < 1e-9
    cm, om = make_ctx(prob, precision=ptp.PTP_MIXED, coarse_steps=coarse_steps)
    for scale in (1.0, 1e-12):   # the float cycle is scale-free
        rm = cm.periodic_solve_dev(cuda(B * scale), X, 8, om)
        assert rm < 1e-3
        assert rel(X.cpu().numpy() / scale, ref) < 1e-3


# ---------------------------------------------------------------------------
# a8: the fixed-point solve, FP64 and mixed, against the oracle's limit
# ---------------------------------------------------------------------------

def _oracle_solution(prob, tol=1e-13):
    d = P.assemble(prob)
    res = P.fixed_point(prob, d, tol=tol, max_it=50000)
    assert res.converged
    return d, res.U


@pytest.mark.parametrize("precision,tol,bar", [("fp64", 1e-13, 1e-10), ("mixed", 1e-11, 1e-8)])
def test_solve_square17(precision, tol, bar):
    prob = W.unit_square_problem(17, 16)
    d, Uo = _oracle_solution(prob)
    prec = ptp.PTP_FP64 if precision == "fp64" else ptp.PTP_MIXED
    c, o = make_ctx(prob, precision=prec, tol=tol, max_outer=20000)
    U, st, rc = c.solve(o)
    assert rc == ptp.PTP_OK and st.converged
    assert rel(U, Uo) < bar
    assert np.linalg.norm(P.residual(prob, d, U)) <= 1.01 * tol * np.linalg.norm(P.source(prob, d))


@pytest.mark.parametrize("precision,tol,bar", [("fp64", 1e-13, 1e-10), ("mixed", 1e-11, 1e-8)])
def test_solve_square33_against_stored_oracle(precision, tol, bar):
    prob = W.config_plain_fp64()
    Uo = np.load(os.path.join(GOLDEN, "square33_N32_oracle.npz"))["U"]
    prec = ptp.PTP_FP64 if precision == "fp64" else ptp.PTP_MIXED
    for graph in (1, 0):
        c, o = make_ctx(prob, precision=prec, tol=tol, max_outer=20000, use_graph=graph)
        U, st, rc = c.solve(o)
        assert rc == ptp.PTP_OK and st.converged
        assert rel(U, Uo) < bar


def test_solve_transformer_and_generic_mesh():
    prob = W.transformer_problem(33, 17, 16)
    d, Uo = _oracle_solution(prob)
    for structured in (True, False):   # GMG on the nested grids / Jacobi on a generic mesh
        c, o = make_ctx(prob, structured, precision=ptp.PTP_FP64, tol=1e-13, max_outer=20000)
        U, st, rc = c.solve(o)
        assert rc == ptp.PTP_OK
        assert rel(U, Uo) < 1e-10


def test_solve_coarse_two_steps_and_half_period_antisymmetry():
    prob = W.unit_square_problem(17, 16, amps=(2000.0,))
    d, Uo = _oracle_solution(prob)
    c, o = make_ctx(prob, precision=ptp.PTP_MIXED, coarse_steps=2, tol=1e-11, max_outer=20000)
    U, st, rc = c.solve(o)
    assert rc == ptp.PTP_OK
    assert rel(U, Uo) < 1e-8
    N = prob.N
    assert np.abs(U[:, N // 2:] + U[:, :N // 2]).max() < 1e-8 * np.abs(U).max()


# ---------------------------------------------------------------------------
# edge and degenerate cases
# ---------------------------------------------------------------------------

def test_single_step_is_the_static_problem():
    """N = 1: u^0 = u^1 removes the mass term, leaving K(u) = f (static)."""
    prob = W.unit_square_problem(17, 1, amps=(3000.0,))
    d, Uo = _oracle_solution(prob)
    c, o = make_ctx(prob, precision=ptp.PTP_FP64, tol=1e-13, max_outer=20000)
    U, st, rc = c.solve(o)
    assert rc == ptp.PTP_OK and rel(U, Uo) < 1e-10


def test_linear_material_converges_in_one_step_and_zero_source():
    prob = W.unit_square_problem(17, 8)
    lin = prob.replace(nonlinear_e=np.zeros(prob.n_tri, np.uint8), nu_linear=prob.nu_max)
    d, Uo = _oracle_solution(lin)
    # 40 V(1,1) cycles per step: the inner periodic solve is exact to rounding
    c, o = make_ctx(lin, precision=ptp.PTP_FP64, tol=1e-9, max_outer=50, vcycles=40, pre_smooth=1, post_smooth=1,
                    omega_t=0.5, coarse_tol=1e-13, coarse_max_it=60)
    U, st, rc = c.solve(o)
    assert rc == ptp.PTP_OK and st.outer_iterations == 1
    assert rel(U, Uo) < 1e-9
    zero = prob.replace(amp=np.zeros(1))
    c, o = make_ctx(zero, precision=ptp.PTP_MIXED, tol=1e-8, max_outer=10)
    U, st, rc = c.solve(o)
    assert rc == ptp.PTP_OK and st.outer_iterations == 0 and np.abs(U).max() == 0.0


def test_not_converged_and_nan_status():
    prob = W.config_plain_fp64()
    c, o = make_ctx(prob, precision=ptp.PTP_MIXED, tol=1e-12, max_outer=7)
    U, st, rc = c.solve(o)
    assert rc == ptp.PTP_ENOTCONV and st.converged == 0 and st.outer_iterations == 7
    assert 0 < st.res_final < st.res0
    n, N, _, _ = c.sizes()
    U0 = np.zeros((n, N))
    U0[5, 3] = np.nan
    with pytest.raises(ptp.PtpError) as e:
        c.solve(o, U0=U0)
    assert e.value.code == ptp.PTP_ENAN


def test_errors_are_reported_not_raised_in_library():
    prob = W.unit_square_problem(9, 6)   # 6 -> 3 steps: no coarsest level with 1 or 2 steps
    c = ptp.Context(0)
    ptp.load_problem(c, prob)
    with pytest.raises(ptp.PtpError) as e:
        c.residual(np.zeros((49, 6)))    # before setup
    assert e.value.code == ptp.PTP_ESTATE
    c.setup(ptp.default_opts())          # residual-only use is fine for any N
    d = P.assemble(prob)
    U = np.random.default_rng(6).normal(size=(49, 6))
    assert rel(c.residual(U)[0], P.residual(prob, d, U)) < 1e-13
    with pytest.raises(ptp.PtpError) as e:
        c.solve()
    assert e.value.code == ptp.PTP_EINVAL
    bad = ptp.Context(0)
    with pytest.raises(ptp.PtpError) as e:
        bad.set_time(-1.0, 4)
    assert e.value.code == ptp.PTP_EINVAL


# ---------------------------------------------------------------------------
# the benchmark workload at full size (257 x 257 nodes, N = 256, mixed)
# ---------------------------------------------------------------------------

def test_full_size_mixed_solve_meets_tolerance_in_oracle_norm():
    """At full size the oracle cannot solve, but it can evaluate: its own
    residual of the GPU iterate must meet the stopping rule, sampled nodes
    of the GPU residual must match it, and the limit must be antisymmetric
    over half a period."""
    prob = W.config_mixed(0)
    d = P.assemble(prob)
    c, o = make_ctx(prob, precision=ptp.PTP_MIXED, tol=1e-8, max_outer=6000)
    n, N, _, _ = c.sizes()
    U = torch.zeros((n, N), dtype=torch.float64, device="cuda")
    st, rc = c.solve_dev(U, o)
    assert rc == ptp.PTP_OK and st.converged
    Uh = U.cpu().numpy()
    F = P.source(prob, d)
    Ro = P.residual(prob, d, Uh, F)
    assert np.linalg.norm(Ro) <= 1.001e-8 * np.linalg.norm(F)
    R = torch.empty_like(U)
    c.residual_dev(U, R)
    rng = np.random.default_rng(5)
    rows = rng.choice(n, size=64, replace=False)
    Rs = R.cpu().numpy()[rows]
    assert np.abs(Rs - Ro[rows]).max() <= 1e-12 * np.abs(F).max()
    assert np.abs(Uh[:, N // 2:] + Uh[:, :N // 2]).max() <= 1e-6 * np.abs(Uh).max()


@pytest.mark.parametrize("precision,tol,bar", [("fp64", 1e-13, 1e-10), ("mixed", 1e-11, 1e-8)])
def test_unstructured_delaunay_mesh(precision, tol, bar):
    """A seeded random Delaunay mesh (no grid structure: Jacobi-preconditioned
    PCG, rows of up to a dozen entries on the CSR path): residual and
    converged solution against the oracle."""
    prob = W.delaunay_problem(300, 8, seed=1, amp=2000.0)
    d = P.assemble(prob)
    prec = ptp.PTP_FP64 if precision == "fp64" else ptp.PTP_MIXED
    c, o = make_ctx(prob, precision=prec, tol=tol, max_outer=20000)
    U = np.random.default_rng(7).normal(scale=0.05, size=(d.n, d.N))
    assert rel(c.residual(U)[0], P.residual(prob, d, U)) < 1e-13
    Us, st, rc = c.solve(o)
    assert rc == ptp.PTP_OK
    ref = P.fixed_point(prob, d, tol=1e-13, max_it=50000)
    assert rel(Us, ref.U) < bar
