"""P1 finite elements on triangles for the 2D model of Section 4.

The spatial model is  sigma d_t u - div(nu(|grad u|) grad u) = j  with
homogeneous Dirichlet data (Section 4, "Test problem"), discretised by
piecewise linear elements ("Simulation setup").  Everything here is fp64 and
written for clarity, not speed.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


_GEOM_CACHE: dict = {}


def p1_geometry(xy: np.ndarray, tri: np.ndarray):
    """Element areas |T| and the constant gradients of the three hat functions
    (memoised per mesh; the arrays are treated as immutable).

    Textbook definition: with the affine map x = p0 + B xi, B = [p1-p0, p2-p0],
    the reference hat functions 1-xi-eta, xi, eta have gradients
    (-1,-1), (1,0), (0,1); physical gradients are B^{-T} times those.
    Returns area (n_tri,) and grad (n_tri, 3, 2).
    """
    key = (xy.__array_interface__["data"][0], xy.shape, tri.__array_interface__["data"][0], tri.shape)
    hit = _GEOM_CACHE.get(key)
    if hit is not None and hit[0] is xy and hit[1] is tri:
        return hit[2], hit[3]
    p = xy[tri]                                   # (n_tri, 3, 2)
    B = np.stack([p[:, 1] - p[:, 0], p[:, 2] - p[:, 0]], axis=2)  # columns
    detB = np.linalg.det(B)
    if np.any(detB <= 0):
        raise ValueError("triangles must be counter-clockwise and non-degenerate")
    ref = np.array([[-1.0, -1.0], [1.0, 0.0], [0.0, 1.0]])       # (3, 2)
    BinvT = np.linalg.inv(B).transpose(0, 2, 1)                   # (n_tri, 2, 2)
    grad = np.einsum("eab,jb->eja", BinvT, ref)                   # (n_tri, 3, 2)
    if len(_GEOM_CACHE) > 8:
        _GEOM_CACHE.clear()
    _GEOM_CACHE[key] = (xy, tri, 0.5 * detB, grad)
    return 0.5 * detB, grad


def stiffness(xy, tri, coef_e):
    """A_ij = sum_T coef_T |T| grad(phi_i).grad(phi_j)  (full node set, CSR)."""
    area, grad = p1_geometry(xy, tri)
    n = xy.shape[0]
    loc = np.einsum("e,eia,eja->eij", coef_e * area, grad, grad)
    rows = np.repeat(tri, 3, axis=1).ravel()
    cols = np.tile(tri, (1, 3)).ravel()
    return sp.csr_matrix((loc.ravel(), (rows, cols)), shape=(n, n))


def mass(xy, tri, sigma_e):
    """Consistent P1 mass  M_ij = sum_T sigma_T |T|/12 (1 + delta_ij)."""
    area, _ = p1_geometry(xy, tri)
    n = xy.shape[0]
    ref = (np.ones((3, 3)) + np.eye(3)) / 12.0
    loc = (sigma_e * area)[:, None, None] * ref[None]
    rows = np.repeat(tri, 3, axis=1).ravel()
    cols = np.tile(tri, (1, 3)).ravel()
    return sp.csr_matrix((loc.ravel(), (rows, cols)), shape=(n, n))


def restrict(Mat, free):
    """Rows/columns of the free (non-Dirichlet) nodes."""
    return Mat[free][:, free].tocsr()


def nu_law(s2, nu_min, nu_max, s_sat):
    """Reluctivity of the iron as a function of s^2 = |grad u|^2:
    nu = nu_min + (nu_max - nu_min) s^2 / (s^2 + s_sat^2)."""
    return nu_min + (nu_max - nu_min) * s2 / (s2 + s_sat * s_sat)


def dnu_ds2(s2, nu_min, nu_max, s_sat):
    """Derivative of nu with respect to s^2."""
    c = s_sat * s_sat
    return (nu_max - nu_min) * c / (s2 + c) ** 2


def exp_law(s2, a, b, c, d):
    """Reluctivity of the paper's transformer materials (Section 4):
    nu = a min(exp(b s^2), c) + d, s^2 = |grad u|^2.  Where exp(b s^2)
    overflows to inf the minimum is c, as it should be; the overflow is
    expected and not reported."""
    with np.errstate(over="ignore"):
        return a * np.minimum(np.exp(b * s2), c) + d


def dexp_law_ds2(s2, a, b, c, d):
    """Derivative of exp_law with respect to s^2: a b exp(b s^2) below the
    cap exp(b s^2) < c, 0 above it (the law has a kink at the cap)."""
    with np.errstate(over="ignore", invalid="ignore"):
        e = np.exp(b * s2)
        return np.where(e < c, a * b * e, 0.0)


def _law_columns(prob, ndim):
    """The exponential-law constants a, b, c, d per element, shaped to
    broadcast against an (n_tri, ...) array with `ndim` dimensions."""
    sh = (-1,) + (1,) * (ndim - 1)
    return [prob.law_abcd[:, k].reshape(sh) for k in range(4)]


def element_nu(prob, s2):
    """nu per element: the nonlinear law on iron, nu_linear elsewhere.
    s2 has shape (n_tri, ...)."""
    iron = prob.nonlinear_e.astype(bool).reshape((-1,) + (1,) * (s2.ndim - 1))
    if prob.law_abcd is not None:
        law = exp_law(s2, *_law_columns(prob, s2.ndim))
    else:
        law = nu_law(s2, prob.nu_min, prob.nu_max, prob.s_sat)
    return np.where(iron, law, prob.nu_linear)


def element_dnu_ds2(prob, s2):
    """d nu / d s^2 per element (0 on linear elements).  s2: (n_tri, ...)."""
    iron = prob.nonlinear_e.astype(bool).reshape((-1,) + (1,) * (s2.ndim - 1))
    if prob.law_abcd is not None:
        dn = dexp_law_ds2(s2, *_law_columns(prob, s2.ndim))
    else:
        dn = dnu_ds2(s2, prob.nu_min, prob.nu_max, prob.s_sat)
    return np.where(iron, dn, 0.0)


def element_gradients(prob, u_full):
    """g_T = sum_j u_j grad(phi_j) for every element and every column of
    u_full (n_nodes, ...).  Returns (n_tri, 2, ...)."""
    _, grad = p1_geometry(prob.xy, prob.tri)
    uT = u_full[prob.tri]                          # (n_tri, 3, ...)
    return np.einsum("eja,ej...->ea...", grad, uT)


def K_apply(prob, u_full):
    """Nonlinear operator of Section 4:  K(u)_i = sum_T nu(|g_T|) |T| g_T . grad(phi_i).

    u_full: (n_nodes, ...) with the Dirichlet nodes set to zero (or to any
    boundary values when testing on the full node set).  One-point quadrature
    is exact because g_T is constant on T.
    """
    area, grad = p1_geometry(prob.xy, prob.tri)
    g = element_gradients(prob, u_full)                       # (n_tri, 2, ...)
    s2 = np.sum(g * g, axis=1)                                # (n_tri, ...)
    nu = element_nu(prob, s2)
    flux = g * (nu * area.reshape((-1,) + (1,) * (s2.ndim - 1)))[:, None]
    contrib = np.einsum("eja,ea...->ej...", grad, flux)        # (n_tri, 3, ...)
    return scatter_matrix(prob) @ contrib.reshape((-1,) + u_full.shape[1:])


def scatter_matrix(prob):
    """0/1 matrix summing element-vertex contributions into nodes
    (row = node id, column = 3*element + local vertex); memoised."""
    key = ("scatter", prob.tri.__array_interface__["data"][0], prob.tri.shape, prob.n_nodes)
    hit = _GEOM_CACHE.get(key)
    if hit is not None and hit[0] is prob.tri:
        return hit[1]
    m = prob.tri.size
    S = sp.csr_matrix((np.ones(m), (prob.tri.ravel(), np.arange(m))), shape=(prob.n_nodes, m))
    _GEOM_CACHE[key] = (prob.tri, S)
    return S


def energy(prob, u_full):
    """Magnetic co-energy E(u) = sum_T |T|/2 W(|g_T|^2) with W' = nu, so that
    grad E = K(u).  For the iron law W(x) = nu_max x - (nu_max-nu_min) c ln(1+x/c),
    c = s_sat^2; for the exponential law W(x) = (a/b)(exp(b min(x, x_c)) - 1)
    + a c max(x - x_c, 0) + d x with x_c = ln(c)/b; for linear elements
    W(x) = nu_linear x.  Used only to pin K."""
    area, _ = p1_geometry(prob.xy, prob.tri)
    g = element_gradients(prob, u_full)
    x = np.sum(g * g, axis=1)
    if prob.law_abcd is not None:
        # W(x) = integral of a min(exp(b y), c) + d over [0, x]
        iron = prob.nonlinear_e.astype(bool)
        a, b, cc, d = (np.where(iron, prob.law_abcd[:, k], 1.0) for k in range(4))
        xc = np.log(cc) / b
        below = a / b * np.expm1(b * np.minimum(x, xc))
        above = a * cc * np.maximum(x - xc, 0.0)
        W_iron = below + above + d * x
    else:
        c = prob.s_sat ** 2
        W_iron = prob.nu_max * x - (prob.nu_max - prob.nu_min) * c * np.log1p(x / c)
    W_lin = prob.nu_linear * x
    W = np.where(prob.nonlinear_e.astype(bool), W_iron, W_lin)
    return float(np.sum(0.5 * area * W))


def K_jacobian(prob, u_full):
    """Frechet derivative DK(u) (full node set, CSR):
    element block |T| grad(phi)^T [nu I + 2 nu'(s^2) g g^T] grad(phi)."""
    area, grad = p1_geometry(prob.xy, prob.tri)
    g = element_gradients(prob, u_full)                       # (n_tri, 2)
    s2 = np.sum(g * g, axis=1)
    nu = element_nu(prob, s2)
    dnu = element_dnu_ds2(prob, s2)
    D = nu[:, None, None] * np.eye(2)[None] + 2.0 * dnu[:, None, None] * np.einsum("ea,eb->eab", g, g)
    loc = area[:, None, None] * np.einsum("eia,eab,ejb->eij", grad, D, grad)
    rows = np.repeat(prob.tri, 3, axis=1).ravel()
    cols = np.tile(prob.tri, (1, 3)).ravel()
    n = prob.n_nodes
    return sp.csr_matrix((loc.ravel(), (rows, cols)), shape=(n, n))


def coil_load(prob):
    """b_c,i = integral of chi_c phi_i = sum over coil-c elements T containing
    i of |T|/3.  Returns (n_coils, n_nodes)."""
    area, _ = p1_geometry(prob.xy, prob.tri)
    b = np.zeros((prob.n_coils, prob.n_nodes))
    for c in range(prob.n_coils):
        sel = prob.coil_of_elem == c
        np.add.at(b[c], prob.tri[sel].ravel(), np.repeat(area[sel] / 3.0, 3))
    return b
