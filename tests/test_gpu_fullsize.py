"""Named workloads at their full sizes, and the multigrid-in-time depth.

At full size the oracle cannot solve, but it evaluates: its own residual of
the GPU iterate must meet the stopping rule, and the limit must be
antisymmetric over half a period (K is odd and every source satisfies
f(t + T/2) = -f(t)).  The oracle residual is formed in chunks of time columns
to bound host memory."""
import os

import numpy as np
import pytest

import workloads as W
from oracle import adjoint as AD
from oracle import periodic as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
ptp = pytest.importorskip("paper_2502_21013_gb300.ptp")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _ctx(prob, **kw):
    c = ptp.Context(0)
    ptp.load_problem(c, prob)
    o = ptp.default_opts(**kw)
    c.setup(o)
    return c, o


def oracle_residual_norm(prob, d, U, chunk=32):
    """||F - A(U)|| by the oracle, chunk by chunk of time columns."""
    F = P.source(prob, d)
    N = d.N
    tot = 0.0
    for j0 in range(0, N, chunk):
        cols = np.arange(j0, min(N, j0 + chunk))
        prev = (cols - 1) % N
        dU = (U[:, cols] - U[:, prev]) / d.tau
        R = F[:, cols] - d.M @ dU - P.K_free(prob, d, U[:, cols])
        tot += float(np.sum(R * R))
    return np.sqrt(tot), float(np.linalg.norm(F))


@pytest.mark.parametrize("levels", [2, 3, 0])
def test_time_hierarchy_depth_two_level_to_full(levels):
    """config 2's two-level to log2(N)-level sweep, on the 33x33, N = 32 case:
    every depth converges to the oracle's solution."""
    prob = W.config_plain_fp64()
    Uo = np.load(os.path.join(GOLDEN, "square33_N32_oracle.npz"))["U"]
    c, o = _ctx(prob, precision=ptp.PTP_MIXED, time_levels=levels, tol=1e-11, max_outer=20000, coarse_cycles=12)
    U, st, rc = c.solve(o)
    assert rc == ptp.PTP_OK
    assert st.time_levels == (levels if levels else 6)
    assert np.linalg.norm(U - Uo) / np.linalg.norm(Uo) < 1e-8


def test_transformer_full_size_mixed():
    """1025x513 nodes (1 048 576 triangles), N = 512, mixed, tol 1e-8."""
    prob = W.config_transformer()
    d = P.assemble(prob)
    c, o = _ctx(prob, precision=ptp.PTP_MIXED, tol=1e-8, max_outer=8000)
    U = torch.zeros((prob.n_free, prob.N), dtype=torch.float64, device="cuda")
    st, rc = c.solve_dev(U, o)
    assert rc == ptp.PTP_OK and st.converged
    Uh = U.cpu().numpy()
    del U
    r, f = oracle_residual_norm(prob, d, Uh)
    assert r <= 1.001e-8 * f
    N = prob.N
    assert np.abs(Uh[:, N // 2:] + Uh[:, :N // 2]).max() <= 1e-6 * np.abs(Uh).max()


def test_adjoint_full_size_fp64():
    """257x257, N = 256, two coils, log-normal iron conductivity, FP64 states:
    J matches the oracle's J of the GPU state, and dJ/d(amp_1) matches a
    central difference (h = 1e-6 relative) of GPU solves.  The states are
    solved to 1e-12: the double residual of this workload bottoms out at
    2.5e-13 relative (its rounding floor, reached by FP64 and mixed alike),
    and 1e-12 / h keeps the difference quotient accurate to about 1e-6."""
    prob = W.config_adjoint(0)
    d = P.assemble(prob)
    opts = dict(precision=ptp.PTP_FP64, tol=1e-12, max_outer=20000)
    c, o = _ctx(prob, **opts)
    U = torch.zeros((prob.n_free, prob.N), dtype=torch.float64, device="cuda")
    st, rc = c.solve_dev(U, o)
    assert rc == ptp.PTP_OK
    J, damp, dnu, dsig, st2, rc2 = c.adjoint_gradient_dev(U, o)
    assert rc2 == ptp.PTP_OK
    Jo = AD.objective(prob, d, U.cpu().numpy())
    assert abs(J - Jo) <= 1e-12 * abs(Jo)
    assert np.all(np.isfinite(dsig.cpu().numpy())) and np.all(np.isfinite(dnu))

    def J_of(amp0):
        p = prob.replace(amp=np.array([amp0, prob.amp[1]]))
        cc, oo = _ctx(p, **opts)
        Uc = torch.zeros((p.n_free, p.N), dtype=torch.float64, device="cuda")
        s, r = cc.solve_dev(Uc, oo)
        assert r == ptp.PTP_OK
        return cc.loss_dev(Uc)

    h = 1e-6 * abs(prob.amp[0])
    fd = (J_of(prob.amp[0] + h) - J_of(prob.amp[0] - h)) / (2 * h)
    assert abs(fd - damp[0]) <= 1e-5 * abs(fd)


def test_newton_full_size_mixed():
    """The bench workload (257x257, N = 256) by Newton's method (M2) to 1e-8:
    the oracle's residual of the iterate meets the stopping rule, the limit is
    half-period antisymmetric, and it agrees with the fixed point's limit."""
    prob = W.config_mixed(0)
    d = P.assemble(prob)
    c, o = _ctx(prob, precision=ptp.PTP_MIXED, tol=1e-8, max_outer=40)
    U, st, rc = c.newton_solve(o)
    assert rc == ptp.PTP_OK and st.outer_iterations <= 30
    r, fn = oracle_residual_norm(prob, d, U)
    assert r <= 1.05e-8 * fn
    N = prob.N
    assert np.abs(U[:, N // 2:] + U[:, :N // 2]).max() <= 1e-6 * np.abs(U).max()
    Uf, st2, rc2 = c.solve(ptp.default_opts(precision=ptp.PTP_MIXED, tol=1e-8, max_outer=6000))
    assert rc2 == ptp.PTP_OK
    assert np.linalg.norm(U - Uf) <= 1e-5 * np.linalg.norm(Uf)


def test_dft_two_level_full_size_mixed():
    """Two-level multigrid in time with the DFT coarse solve on 128 steps, the
    bench workload to 1e-8: the oracle's residual meets the stopping rule."""
    prob = W.config_mixed(0)
    d = P.assemble(prob)
    c, o = _ctx(prob, precision=ptp.PTP_MIXED, tol=1e-8, max_outer=6000, coarse_solver=1, time_levels=2)
    U, st, rc = c.solve(o)
    assert rc == ptp.PTP_OK and st.time_levels == 2
    r, fn = oracle_residual_norm(prob, d, U)
    assert r <= 1.05e-8 * fn
