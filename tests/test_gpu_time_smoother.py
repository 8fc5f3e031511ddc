"""The automatic time smoother on the GPU: set-up's inverse-iteration
estimate of lambda_min(L, M) against scipy's generalised eigenvalue of the
oracle's assembled matrices, the choice it makes (the host model's choice at
0.9 tau lambda_min), and convergence of solves that need the robust cycle
(the paper's transformer, kappa_min ~ 1e-3) and that take the cheap one."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as W
from oracle import periodic as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
ptp = pytest.importorskip("paper_2502_21013_gb300.ptp")


def lambda_min(prob):
    d = P.assemble(prob)
    lu = spla.splu(d.L.tocsc())
    op = spla.LinearOperator(d.L.shape, matvec=lambda x: lu.solve(d.M @ x))
    mu = spla.eigs(op, k=1, which="LM", return_eigenvectors=False, tol=1e-12)
    return 1.0 / abs(mu[0]), d


# (name, problem, expected choice: "fast" = V(1,0) with omega 0.95, "robust" =
# damping <= 0.6, where V(1,0) with omega 0.95 would amplify the slow modes)
CASES = [
    ("square33_N32", lambda: W.unit_square_problem(33, 32), "fast"),
    ("transformer65x33_N32", lambda: W.transformer_problem(65, 33, 32), None),
    ("paper41x53_N16", lambda: W.paper_transformer_problem(41, 53, 16), "robust"),
]


@pytest.mark.parametrize("name,make,expect", CASES, ids=[c[0] for c in CASES])
def test_kappa_estimate_and_choice(name, make, expect):
    prob = make()
    lam, d = lambda_min(prob)
    c = ptp.Context(0)
    ptp.load_problem(c, prob)
    o = ptp.default_opts(precision=ptp.PTP_MIXED, tol=1e-8, max_outer=3)
    c.setup(o)
    U = torch.zeros((prob.n_free, prob.N), dtype=torch.float64, device="cuda")
    st, rc = c.solve_dev(U, o)
    assert rc in (ptp.PTP_OK, ptp.PTP_ENOTCONV)
    kappa = d.tau * lam
    assert st.kappa_min == pytest.approx(kappa, rel=1e-3)
    levels = [prob.N >> k for k in range(st.time_levels)]
    post, omega, _ = ptp.choose_time_smoother(levels, 0.9 * st.kappa_min)
    assert (st.post_smooth, st.omega_t) == (post, omega)
    if expect == "fast":
        assert (st.post_smooth, st.omega_t) == (0, 0.95)
    elif expect == "robust":
        assert st.omega_t <= 0.6
        assert ptp.time_cycle_rho(levels, 0.9 * st.kappa_min, 1, 0, 0.95) > 1.0


def test_explicit_values_are_kept():
    prob = W.unit_square_problem(17, 8)
    c = ptp.Context(0)
    ptp.load_problem(c, prob)
    o = ptp.default_opts(precision=ptp.PTP_FP64, tol=1e-8, max_outer=2, post_smooth=1, omega_t=0.6)
    c.setup(o)
    U = torch.zeros((prob.n_free, prob.N), dtype=torch.float64, device="cuda")
    st, rc = c.solve_dev(U, o)
    assert (st.post_smooth, st.omega_t, st.kappa_min) == (1, 0.6, 0.0)


@pytest.mark.parametrize("precision,tol,bar", [(ptp.PTP_FP64, 1e-11, 1e-9), (ptp.PTP_MIXED, 1e-10, 1e-8)])
def test_paper_transformer_converges_with_the_default_cycle(precision, tol, bar):
    """With the default options (one PCG iteration per spatial solve) the
    paper's transformer, whose slow modes have kappa ~ 1e-3, reaches the
    oracle's fixed point."""
    prob = W.paper_transformer_problem(41, 53, 16)
    d = P.assemble(prob)
    ref = P.fixed_point(prob, d, tol=1e-13, max_it=500)
    assert ref.converged
    c = ptp.Context(0)
    ptp.load_problem(c, prob)
    o = ptp.default_opts(precision=precision, tol=tol, max_outer=20000)
    c.setup(o)
    U, st, rc = c.solve(o)
    assert rc == ptp.PTP_OK
    assert st.omega_t <= 0.6
    assert np.linalg.norm(U - ref.U) / np.linalg.norm(ref.U) < bar
