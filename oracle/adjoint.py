"""Discrete adjoint of the period-averaged eddy-current loss (tiny meshes).

Objective, at the solution U of Problem 1 (A(U) = F):
    J = (1/N) sum_n sum_{e in iron} sigma_e (d_tau u^n)_e^T M1_e (d_tau u^n)_e,
with d_tau u^n = (u^n - u^{n-1})/tau, u^0 = u^N, and M1_e the unit-conductivity
consistent P1 element mass |T|/12 (1 + delta_ab), so that each term is the
integral of sigma |d_tau u|^2 over the element.

Parameters p: the coil amplitudes amp_c, the reluctivity parameters
(nu_min, nu_max, s_sat) of the iron law and the conductivity sigma_e of
every element.  With G(U, p) = A(U; p) - F(p) = 0, the implicit-function
theorem gives
    dJ/dp = dJ/dp|_U - lambda^T dG/dp,   (dG/dU)^T lambda = (dJ/dU)^T,
where dG/dU is the space-time Jacobian of A (diagonal blocks M/tau + DK(u^n),
cyclic sub-diagonal -M/tau), so the adjoint runs backward in time with
lambda^{N+1} = lambda^1.  The fixed point's K_hat = nu_max A does not enter
A(U), so nu_max acts through the reluctivity law only; nu_linear of the
non-iron elements is not a parameter.

Everything is fp64; the adjoint system is solved by a sparse LU of the full
space-time Jacobian (tiny sizes only).
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem
from . import periodic as P


def loss_mass(prob, disc):
    """M_J = sum over iron elements of sigma_e M1_e, free nodes only."""
    sig = np.where(prob.nonlinear_e.astype(bool), prob.sigma_e, 0.0)
    return fem.restrict(fem.mass(prob.xy, prob.tri, sig), disc.free)


def objective(prob, disc, U):
    d = (U - np.roll(U, 1, axis=1)) / disc.tau
    MJ = loss_mass(prob, disc)
    return float(np.sum(d * (MJ @ d))) / disc.N


def objective_grad_U(prob, disc, U):
    """dJ/du^n = (2/(N tau)) M_J (d^n - d^{n+1}), d^{N+1} = d^1."""
    d = (U - np.roll(U, 1, axis=1)) / disc.tau
    MJd = loss_mass(prob, disc) @ d
    return 2.0 / (disc.N * disc.tau) * (MJd - np.roll(MJd, -1, axis=1))


def adjoint_solve(prob, disc, U, g):
    """(dA/dU)^T lambda = g with the space-time Jacobian of periodic.jacobian."""
    Jm = P.jacobian(prob, disc, U).T.tocsc()
    return spla.spsolve(Jm, g.ravel()).reshape(g.shape)


def dnu_dtheta(prob, s2):
    """Partial derivatives of the iron law nu(s^2) with respect to
    (nu_min, nu_max, s_sat).  Returns (3, ...)."""
    c = prob.s_sat ** 2
    q = s2 / (s2 + c)
    d_min = 1.0 - q
    d_max = q
    d_sat = -(prob.nu_max - prob.nu_min) * s2 * 2.0 * prob.s_sat / (s2 + c) ** 2
    return np.stack([d_min, d_max, d_sat])


def parameter_gradients(prob, disc, U, lam):
    """dJ/d(amp), dJ/d(nu_min, nu_max, s_sat), dJ/d(sigma_e) from U and lambda."""
    N, tau = disc.N, disc.tau
    # coils: dG/d amp_c = -f_c (unit-amplitude source of coil c)
    t = tau * np.arange(1, N + 1)
    d_amp = np.zeros(prob.n_coils)
    for c in range(prob.n_coils):
        fc = np.sin(2 * math.pi * t[None, :] / prob.T + prob.phase[c]) * disc.b[c][:, None]
        d_amp[c] = float(np.sum(lam * fc))
    # reluctivity parameters: dG/dtheta = sum_iron |T| dnu/dtheta g . grad(phi_i)
    area, grad = fem.p1_geometry(prob.xy, prob.tri)
    Uf = P.lift(prob, disc, U)
    Lf = P.lift(prob, disc, lam)
    g = fem.element_gradients(prob, Uf)            # (n_tri, 2, N)
    h = fem.element_gradients(prob, Lf)
    s2 = np.sum(g * g, axis=1)                      # (n_tri, N)
    gh = np.sum(g * h, axis=1)
    iron = prob.nonlinear_e.astype(bool)
    dn = dnu_dtheta(prob, s2)                       # (3, n_tri, N)
    d_nu = -np.sum(dn[:, iron, :] * (area[iron, None] * gh[iron])[None], axis=(1, 2))
    # conductivities: dJ/dsigma_e|_U - lambda^T M1_e (u^n - u^{n-1})/tau
    du = (Uf - np.roll(Uf, 1, axis=1)) / tau        # (n_nodes, N)
    M1 = (np.ones((3, 3)) + np.eye(3)) / 12.0
    de = du[prob.tri]                               # (n_tri, 3, N)
    le = Lf[prob.tri]
    quad_u = np.einsum("eaN,ab,ebN->e", de, M1, de) * area
    quad_lu = np.einsum("eaN,ab,ebN->e", le, M1, de) * area
    d_sigma = np.where(iron, quad_u / N, 0.0) - quad_lu
    return d_amp, d_nu, d_sigma


def gradient(prob, disc=None, U=None, tol=1e-14):
    """J and its gradients at the solution of Problem 1 (solved by Newton)."""
    if disc is None:
        disc = P.assemble(prob)
    if U is None:
        U, _ = P.newton(prob, disc, tol=tol)
    g = objective_grad_U(prob, disc, U)
    lam = adjoint_solve(prob, disc, U, g)
    d_amp, d_nu, d_sigma = parameter_gradients(prob, disc, U, lam)
    return objective(prob, disc, U), d_amp, d_nu, d_sigma, lam
