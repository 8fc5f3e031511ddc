"""Pins of the oracle's adjoint gradient against central finite differences
of J(U(p)), with U re-solved to machine precision by Newton for every
perturbed parameter (an independent route to the same derivative)."""
import numpy as np
import pytest

import workloads as W
from oracle import adjoint as AD
from oracle import periodic as P


def _problem(T=1.0, s_sat=1.0):
    prob = W.config_adjoint(0, n=7, N=4)
    # strong coils so the iron law is exercised on both sides of s_sat
    return prob.replace(amp=np.array([7000.0, 4500.0]), phase=np.array([0.0, 0.7]), T=T, s_sat=s_sat)


# the period and s_sat enter the time derivative, the source and the law:
# a second case away from 1 keeps a misplaced T or s_sat from cancelling
CASES = [(1.0, 1.0), (0.5, 0.7)]


def _J(prob):
    d = P.assemble(prob)
    U, rel = P.newton(prob, d, tol=1e-15)
    return AD.objective(prob, d, U)


def test_objective_closed_form():
    """U^n = n w with w = 1 on every free node: the periodic difference is
    w / tau for n >= 2 and (1 - N) w / tau for n = 1, and w^T M_J w is the sum
    of sigma_e |T_e| over the iron elements (all inside the domain, and a
    consistent element mass sums to the element area), so
    J = (1/N) [(N - 1) + (N - 1)^2] w^T M_J w / tau^2 = (N - 1) sum sigma_e |T_e| / tau^2."""
    for T, s_sat in CASES:
        prob = _problem(T, s_sat)
        d = P.assemble(prob)
        U = np.outer(np.ones(d.n), np.arange(1, d.N + 1, dtype=np.float64))
        iron = prob.nonlinear_e.astype(bool)
        h = 1.0 / 6.0                                   # 7 x 7 nodes on the unit square
        ref = (d.N - 1) * np.sum(prob.sigma_e[iron]) * (h * h / 2) / (T / d.N) ** 2
        assert AD.objective(prob, d, U) == pytest.approx(ref, rel=1e-12)


@pytest.mark.parametrize("T,s_sat", CASES)
def test_objective_gradient_in_U_matches_differences(T, s_sat):
    prob = _problem(T, s_sat)
    d = P.assemble(prob)
    rng = np.random.default_rng(0)
    U = rng.normal(scale=0.05, size=(d.n, d.N))
    V = rng.normal(size=(d.n, d.N))
    g = AD.objective_grad_U(prob, d, U)
    h = 1e-6
    fd = (AD.objective(prob, d, U + h * V) - AD.objective(prob, d, U - h * V)) / (2 * h)
    assert abs(fd - np.sum(g * V)) <= 1e-7 * abs(fd)


@pytest.mark.parametrize("T,s_sat", CASES)
def test_adjoint_gradient_matches_central_differences(T, s_sat):
    prob = _problem(T, s_sat)
    J0, d_amp, d_nu, d_sigma, _ = AD.gradient(prob)
    assert J0 > 0
    d = P.assemble(prob)
    U, _ = P.newton(prob, d, tol=1e-15)
    s = np.sqrt((np.sum(__import__("oracle").fem.element_gradients(prob, P.lift(prob, d, U))[:, :, :] ** 2, axis=1)))
    iron = prob.nonlinear_e.astype(bool)
    assert s[iron].max() > prob.s_sat  # nonlinear regime
    checks = []
    for c in range(prob.n_coils):
        checks.append((lambda p, v, c=c: p.replace(amp=np.where(np.arange(p.n_coils) == c, v, p.amp)),
                       prob.amp[c], d_amp[c]))
    for k, name in enumerate(("nu_min", "nu_max", "s_sat")):
        checks.append((lambda p, v, name=name: p.replace(**{name: v}), getattr(prob, name), d_nu[k]))
    rng = np.random.default_rng(1)
    elems = list(rng.choice(np.flatnonzero(iron), 3, replace=False)) + \
        list(rng.choice(np.flatnonzero(~iron), 2, replace=False))
    for e in elems:
        def setter(p, v, e=e):
            sig = p.sigma_e.copy()
            sig[e] = v
            return p.replace(sigma_e=sig)
        checks.append((setter, prob.sigma_e[e], d_sigma[e]))
    for setter, p0, grad in checks:
        h = 1e-6 * max(1.0, abs(p0))
        fd = (_J(setter(prob, p0 + h)) - _J(setter(prob, p0 - h))) / (2 * h)
        assert abs(fd - grad) <= 1e-5 * max(abs(fd), 1e-3 * abs(J0)), (p0, fd, grad)
