"""Pins of the oracle's adjoint gradient against central finite differences
of J(U(p)), with U re-solved to machine precision by Newton for every
perturbed parameter (an independent route to the same derivative)."""
import numpy as np
import pytest

import workloads as W
from oracle import adjoint as AD
from oracle import periodic as P


def _problem():
    prob = W.config_adjoint(0, n=7, N=4)
    # strong coils so the iron law is exercised on both sides of s_sat
    return prob.replace(amp=np.array([7000.0, 4500.0]), phase=np.array([0.0, 0.7]))


def _J(prob):
    d = P.assemble(prob)
    U, rel = P.newton(prob, d, tol=1e-15)
    return AD.objective(prob, d, U)


def test_objective_gradient_in_U_matches_differences():
    prob = _problem()
    d = P.assemble(prob)
    rng = np.random.default_rng(0)
    U = rng.normal(scale=0.05, size=(d.n, d.N))
    V = rng.normal(size=(d.n, d.N))
    g = AD.objective_grad_U(prob, d, U)
    h = 1e-6
    fd = (AD.objective(prob, d, U + h * V) - AD.objective(prob, d, U - h * V)) / (2 * h)
    assert abs(fd - np.sum(g * V)) <= 1e-7 * abs(fd)


def test_adjoint_gradient_matches_central_differences():
    prob = _problem()
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
