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


def _perturbed_J(c, prob, U_star, opts_setup):
    """J(U(p)) for a perturbed problem: U(p) by Newton's method (M2) started
    from the unperturbed solution U_star, stopped at ||F - A(U)|| <= 5e-13 ||F||
    (just above the double residual's rounding floor of this workload).  The
    solution of Problem 1 is unique (Theorem 2), so the solver that reaches it
    does not matter; a warm-started Newton solve takes a few steps."""
    ptp.load_problem(c, prob)
    c.setup(opts_setup)
    zero = torch.zeros_like(U_star)
    f = c.residual_dev(zero)
    r0 = c.residual_dev(U_star)
    o = ptp.default_opts(precision=ptp.PTP_MIXED, tol=min(0.5, 5e-13 * f / r0), max_outer=30)
    U = torch.empty_like(U_star)
    st, rc = c.newton_solve_dev(U, o, U0=U_star)
    assert rc == ptp.PTP_OK, (rc, st.res_final / f)
    return c.loss_dev(U)


def test_adjoint_full_size_every_parameter_class():
    """257x257, N = 256, two coils, log-normal iron conductivity, FP64 states:
    J matches the oracle's J of the GPU state, and the adjoint gradient
    matches finite differences of J(U(p)) on the GPU for both coil
    amplitudes, nu_min, nu_max, s_sat and a seeded sample of 16 iron
    conductivities, each to 1e-5 relative.

    Steps: the amplitudes by central differences with h = 1e-6 |p|.  nu_min,
    nu_max, s_sat (h = 1e-3 |p|) and sigma_e (h = 2e-2 sigma_e) by central
    differences at h and h/2 combined by Richardson extrapolation, which
    removes the h^2 term.  A single element's conductivity moves J by 1e-7 to
    1e-5 of itself per unit relative change, while J of a state solved to the
    double residual's floor (2.5e-13 relative on this workload) reproduces to
    about eps = 5e-12 of itself.  The Richardson value (4 D(h/2) - D(h)) / 3
    of the central differences D(h/2) = (J+ - J-) / h and D(h) =
    (J++ - J--) / (2 h) carries at most (4 * 2 + 1) / 3 = 3 eps J / h of that
    noise; so each sampled sigma_e is checked to 1e-5 relative plus the floor
    3 eps J / h, and the directional derivative along a
    seeded random combination of every iron conductivity, whose change of J
    is far above the noise, to 1e-5 relative.  The base state is solved to
    1e-12."""
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
    dsig = dsig.cpu().numpy()
    assert np.all(np.isfinite(dsig)) and np.all(np.isfinite(dnu))
    del c

    cf = ptp.Context(0)
    so = ptp.default_opts(precision=ptp.PTP_MIXED)

    def J_at(setter, v):
        return _perturbed_J(cf, setter(prob, v), U, so)

    def central(setter, p0, h):
        return (J_at(setter, p0 + h) - J_at(setter, p0 - h)) / (2 * h)

    def richardson(setter, p0, h):
        return (4 * central(setter, p0, h / 2) - central(setter, p0, h)) / 3

    iron = np.flatnonzero(prob.nonlinear_e)
    sample = np.random.default_rng(2024).choice(iron, 16, replace=False)
    cases = [
        ("amp1", lambda p, v: p.replace(amp=np.array([v, p.amp[1]])), prob.amp[0], damp[0], "central", 1e-6),
        ("amp2", lambda p, v: p.replace(amp=np.array([p.amp[0], v])), prob.amp[1], damp[1], "central", 1e-6),
        ("nu_min", lambda p, v: p.replace(nu_min=v), prob.nu_min, dnu[0], "richardson", 1e-3),
        ("nu_max", lambda p, v: p.replace(nu_max=v), prob.nu_max, dnu[1], "richardson", 1e-3),
        ("s_sat", lambda p, v: p.replace(s_sat=v), prob.s_sat, dnu[2], "richardson", 1e-3),
    ]
    for e in sample:
        cases.append((f"sigma[{e}]", lambda p, v, e=e: p.replace(sigma_e=np.where(np.arange(p.n_tri) == e, v,
                                                                                         p.sigma_e)),
                      prob.sigma_e[e], dsig[e], "richardson", 2e-2))
    # every iron conductivity along one seeded direction v (relative steps):
    # sigma(t) = sigma * (1 + t v), dJ/dt at 0 = sum_e sigma_e v_e dJ/dsigma_e
    v = np.zeros(prob.n_tri)
    v[iron] = np.random.default_rng(7).uniform(-1.0, 1.0, iron.size)
    cases.append(("sigma along v", lambda p, t: p.replace(sigma_e=prob.sigma_e * (1.0 + t * v)), 0.0,
                  float(np.sum(prob.sigma_e * v * dsig)), "richardson", None))
    bad = []
    for name, setter, p0, grad, kind, hrel in cases:
        h = hrel * abs(p0) if hrel is not None else 1e-3
        fd = central(setter, p0, h) if kind == "central" else richardson(setter, p0, h)
        err = abs(fd - grad) / abs(fd)
        floor = 3 * 5e-12 * abs(J) / h if name.startswith("sigma[") else 0.0
        print(f"adjoint FD {name}: adjoint {grad:.10e} FD {fd:.10e} rel. diff {err:.2e} "
              f"(noise floor {floor / abs(fd):.1e} relative)")
        if not abs(fd - grad) <= 1e-5 * abs(fd) + floor:
            bad.append((name, grad, fd, err))
    assert not bad, bad


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
