"""Pins of the CPU oracle against facts that do not come from the oracle.

Each test names the fact it checks: a textbook stencil, a closed form, an
identity of the model, or an independent brute-force solver.  The cases are
chosen so that a dropped term, a wrong sign or index, or a transposed
operand in the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle import fem
from oracle import periodic as P


def _uniform(n, N=4, *, sigma=1.0, nonlinear=True, nu_linear=100.0, amp=50.0):
    prob = W.unit_square_problem(n, N, amps=(amp,))
    ne = prob.n_tri
    return prob.replace(sigma_e=np.full(ne, sigma),
                        nonlinear_e=np.full(ne, 1 if nonlinear else 0, np.uint8),
                        nu_linear=nu_linear)


# --------------------------------------------------------------------------
# Assembly: textbook stencils of P1 on the right-triangle grid
# --------------------------------------------------------------------------

def test_stiffness_is_five_point_laplacian():
    """P1 stiffness on the uniform right-triangle grid is the classical
    5-point stencil (4, -1, -1, -1, -1); the diagonal edges carry 0 because
    the angle opposite them is a right angle."""
    n = 7
    prob = _uniform(n)
    A = fem.stiffness(prob.xy, prob.tri, np.ones(prob.n_tri)).toarray()
    free = prob.interior
    ref = np.zeros((n * n, n * n))
    for j in range(1, n - 1):
        for i in range(1, n - 1):
            k = j * n + i
            ref[k, k] = 4.0
            for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                ref[k, (j + dj) * n + (i + di)] = -1.0
    np.testing.assert_allclose(A[np.ix_(free, free)], ref[np.ix_(free, free)], atol=1e-13)


def test_mass_stencil_and_total():
    """Consistent P1 mass with sigma = 1: row of an interior node has
    h^2/2 on the diagonal and h^2/12 to the six neighbours sharing an edge
    ((+-1,0), (0,+-1), (1,1), (-1,-1)); the sum of all entries is the area."""
    n = 9
    h = 1.0 / (n - 1)
    prob = _uniform(n, sigma=1.0)
    M = fem.mass(prob.xy, prob.tri, prob.sigma_e).toarray()
    assert abs(M.sum() - 1.0) < 1e-13
    j = i = 4
    k = j * n + i
    row = np.zeros(n * n)
    row[k] = h * h / 2
    for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1), (1, 1), (-1, -1)):
        row[(j + dj) * n + (i + di)] = h * h / 12
    np.testing.assert_allclose(M[k], row, atol=1e-15)


def test_degenerate_or_clockwise_triangles_are_rejected():
    """The P1 map needs det B > 0: a zero-area or clockwise triangle has none."""
    xy = np.array([[0.0, 0.0], [1.0, 0.0], [2.0, 0.0], [0.0, 1.0]])
    with pytest.raises(ValueError, match="counter-clockwise"):
        fem.p1_geometry(xy, np.array([[0, 1, 2]]))      # collinear: zero area
    with pytest.raises(ValueError, match="counter-clockwise"):
        fem.p1_geometry(xy, np.array([[0, 3, 1]]))      # clockwise
    area, _ = fem.p1_geometry(xy, np.array([[0, 1, 3]]))
    assert area[0] == 0.5


def test_stiffness_kernel_and_symmetry():
    """The full-node stiffness annihilates constants (rows sum to zero) and
    is symmetric."""
    prob = W.transformer_problem(17, 9, 4)
    A = fem.stiffness(prob.xy, prob.tri, np.linspace(1, 3, prob.n_tri))
    assert abs(A - A.T).max() < 1e-13
    assert np.abs(A @ np.ones(prob.n_nodes)).max() < 1e-12


# --------------------------------------------------------------------------
# Nonlinear operator K
# --------------------------------------------------------------------------

def test_K_vanishes_on_linear_field():
    """For u = a x + b y the gradient is constant, so nu is constant and
    K(u)_i = nu g . sum_T |T| grad(phi_i) = 0 at every interior node."""
    prob = _uniform(9)
    u = 0.3 * prob.xy[:, 0] - 0.7 * prob.xy[:, 1]
    Ku = fem.K_apply(prob, u)
    assert np.abs(Ku[prob.interior]).max() < 1e-12


@pytest.mark.parametrize("s_sat", [1.0, 0.6])
def test_K_is_gradient_of_coenergy(s_sat):
    """K(u) = grad E(u) with E = sum_T |T|/2 W(|g_T|^2), W' = nu, where W is
    the closed-form antiderivative of the reluctivity law (log form).
    Checked by central differences on a random field, mixed materials."""
    prob = W.unit_square_problem(9, 4, s_sat=s_sat)
    rng = np.random.default_rng(3)
    u = np.zeros(prob.n_nodes)
    u[prob.interior] = rng.normal(scale=0.8, size=prob.n_free)
    Ku = fem.K_apply(prob, u)
    h = 1e-6
    for i in prob.interior[::5]:
        e = np.zeros_like(u)
        e[i] = h
        fd = (fem.energy(prob, u + e) - fem.energy(prob, u - e)) / (2 * h)
        assert abs(fd - Ku[i]) <= 1e-7 * max(1.0, abs(Ku[i]))


def test_K_one_node_closed_form():
    """3x3 grid, h = 1/2, single free node c, all elements iron.  Four of the
    six elements at c have |grad phi_c|^2 = 1/h^2 and two (right angle at c)
    have 2/h^2, each of area h^2/2, hence
    K(u_c) = [2 nu(u^2/h^2) + 2 nu(2u^2/h^2)] u_c."""
    prob = W.one_node_problem(4)
    h = 0.5
    for uc in (0.0, 0.1, 0.37, -1.3):
        u = np.zeros(prob.n_nodes)
        u[4] = uc
        nu = lambda s2: fem.nu_law(s2, prob.nu_min, prob.nu_max, prob.s_sat)
        ref = (2 * nu(uc**2 / h**2) + 2 * nu(2 * uc**2 / h**2)) * uc
        assert abs(fem.K_apply(prob, u)[4] - ref) < 1e-12 * max(1, abs(ref))


def test_nu_law_limits():
    """nu(0) = nu_min, nu(s_sat) = (nu_min+nu_max)/2, nu(inf) -> nu_max."""
    assert fem.nu_law(0.0, 1.0, 100.0, 1.0) == 1.0
    assert abs(fem.nu_law(4.0, 1.0, 100.0, 2.0) - 50.5) < 1e-13
    assert abs(fem.nu_law(1e12, 1.0, 100.0, 1.0) - 100.0) < 1e-8


@pytest.mark.parametrize("s_sat", [1.0, 0.6])
def test_K_jacobian_matches_differences(s_sat):
    """DK(u) v equals the central difference of K along v."""
    prob = W.unit_square_problem(9, 4, s_sat=s_sat)
    rng = np.random.default_rng(5)
    u = np.zeros(prob.n_nodes)
    v = np.zeros(prob.n_nodes)
    u[prob.interior] = rng.normal(scale=0.7, size=prob.n_free)
    v[prob.interior] = rng.normal(size=prob.n_free)
    J = fem.K_jacobian(prob, u)
    h = 1e-6
    fd = (fem.K_apply(prob, u + h * v) - fem.K_apply(prob, u - h * v)) / (2 * h)
    np.testing.assert_allclose(J @ v, fd, rtol=1e-6, atol=1e-8)


# --------------------------------------------------------------------------
# Source
# --------------------------------------------------------------------------

def test_coil_load_total_is_coil_area():
    """sum_i b_c,i = integral of chi_c = (number of coil elements) * h^2/2
    on the uniform grid (each element gives |T|/3 to three vertices)."""
    prob = W.config_plain_fp64()
    b = fem.coil_load(prob)
    h = 1.0 / 32
    count = int((prob.coil_of_elem == 0).sum())
    assert count > 0
    assert abs(b.sum() - count * h * h / 2) < 1e-14


@pytest.mark.parametrize("T", [1.0, 0.02])
def test_source_sampling_times(T):
    """f^n is sampled at t^n = n tau, n = 1..N: for one coil with phase 0,
    column N-1 (t = T) is sin(2 pi) b = 0 and column N/4 - 1 is b, whatever
    the period."""
    prob = W.config_plain_fp64().replace(T=T)
    d = P.assemble(prob)
    F = P.source(prob, d)
    b = d.b[0] * prob.amp[0]
    assert np.abs(F[:, -1]).max() < 1e-12 * np.abs(b).max()
    np.testing.assert_allclose(F[:, prob.N // 4 - 1], b, rtol=1e-14, atol=1e-16)


# --------------------------------------------------------------------------
# Exact periodic linear solvers
# --------------------------------------------------------------------------

def test_periodic_solvers_agree_with_dense():
    """Space-time sparse LU, time-DFT and a dense solve of the same
    block-cyclic system agree (odd and even N)."""
    prob = W.unit_square_problem(6, 5)
    d = P.assemble(prob)
    rng = np.random.default_rng(0)
    for N in (5, 6):
        B = rng.normal(size=(d.n, N))
        X0 = P.dense_periodic_solve(d.M, d.L, 0.1, B)
        X1 = P.SpaceTimeLU(d.M, d.L, 0.1, N).solve(B)
        X2 = P.DFTSolver(d.M, d.L, 0.1, N).solve(B)
        np.testing.assert_allclose(X1, X0, rtol=1e-11, atol=1e-13)
        np.testing.assert_allclose(X2, X0, rtol=1e-11, atol=1e-13)


def test_periodic_matrix_structure():
    """The space-time matrix applied to X gives M(x^n - x^{n-1})/tau + K x^n
    with x^0 = x^N, written out column by column."""
    prob = W.unit_square_problem(6, 4)
    d = P.assemble(prob)
    rng = np.random.default_rng(1)
    N, tau = 4, 0.25
    X = rng.normal(size=(d.n, N))
    Y = (P.periodic_matrix(d.M, d.L, tau, N) @ X.ravel()).reshape(X.shape)
    for j in range(N):
        prev = X[:, N - 1] if j == 0 else X[:, j - 1]
        ref = d.M @ (X[:, j] - prev) / tau + d.L @ X[:, j]
        np.testing.assert_allclose(Y[:, j], ref, rtol=1e-13, atol=1e-13)


def test_scalar_periodic_closed_form():
    """One free node, linear material with nu = nu_max (so K = L and the
    fixed point is exact after one step), f^n = a b sin(2 pi n/N).
    Closed form: u^n = Im(c e^{i theta n}), theta = 2 pi/N,
    c = a b / (m (1 - e^{-i theta})/tau + l), m = sigma h^2/2, l = 4 nu_max,
    b = 6 (h^2/2)/3 with h = 1/2."""
    N = 8
    prob = W.one_node_problem(N, nonlinear=False, sigma=10.0, amp=3.0)
    res = P.fixed_point(prob, tol=1e-14, max_it=5)
    h = 0.5
    m = 10.0 * h * h / 2
    l = 4 * prob.nu_max
    b = 6 * (h * h / 2) / 3
    tau = prob.T / N
    th = 2 * math.pi / N
    c = 3.0 * b / (m * (1 - np.exp(-1j * th)) / tau + l)
    ref = np.imag(c * np.exp(1j * th * np.arange(1, N + 1)))
    np.testing.assert_allclose(res.U[0], ref, rtol=1e-13, atol=1e-16)
    assert res.iterations == 1


# --------------------------------------------------------------------------
# Fixed-point iteration (Theorem 3) and its limit (Theorem 2)
# --------------------------------------------------------------------------

def test_one_step_convergence_when_K_is_Khat():
    """nu = nu_max everywhere makes K = K_hat, so eq. (iter1) is the exact
    problem and one step gives the solution."""
    prob = W.unit_square_problem(9, 8)
    prob = prob.replace(nonlinear_e=np.zeros(prob.n_tri, np.uint8), nu_linear=prob.nu_max)
    res = P.fixed_point(prob, tol=1e-13, max_it=3)
    assert res.iterations == 1 and res.converged


def test_fixed_point_matches_newton_tiny():
    """The fixed-point limit equals the solution of A(U) = F obtained by an
    independent Newton solver (unique by Theorem 2); strong nonlinearity
    (large source) so that nu varies across the iron."""
    prob = W.unit_square_problem(7, 6, amps=(4000.0,), coil_boxes=(((0.05, 0.45), (0.2, 0.8)),))
    d = P.assemble(prob)
    Un, rel = P.newton(prob, d, tol=1e-14)
    assert rel < 1e-13
    res = P.fixed_point(prob, d, tol=1e-14, max_it=20000)
    assert res.converged
    err = np.linalg.norm(res.U - Un) / np.linalg.norm(Un)
    assert err < 1e-11
    full = P.lift(prob, d, Un)
    s = np.sqrt((fem.element_gradients(prob, full) ** 2).sum(axis=1))
    iron = prob.nonlinear_e.astype(bool)
    # the solution visits both sides of s_sat in the iron, so nu is nonlinear
    assert s[iron].max() > prob.s_sat > s[iron].min()


def test_manufactured_periodic_solution():
    """Choose U*, set F := A(U*); the iteration recovers U*."""
    prob = W.unit_square_problem(9, 8)
    d = P.assemble(prob)
    x, y = prob.xy[d.free, 0], prob.xy[d.free, 1]
    t = d.tau * np.arange(1, d.N + 1)
    U = np.outer(np.sin(math.pi * x) * np.sin(math.pi * y),
                 np.cos(2 * math.pi * t) + 0.5 * np.sin(4 * math.pi * t)) * 0.8
    F = P.A_apply(prob, d, U)
    res = P.fixed_point(prob, d, F=F, tol=1e-13, max_it=20000)
    assert res.converged
    assert np.linalg.norm(res.U - U) / np.linalg.norm(U) < 1e-11


def test_half_period_antisymmetry_and_contraction():
    """K is odd and f(t + T/2) = -f(t), so the unique solution satisfies
    u^{n+N/2} = -u^n.  Theorem 3 with K_hat = nu_max A: the observed ratio
    ||U^{k+1}-U^k||_Khat / ||U^k-U^{k-1}||_Khat stays below 1 - nu_min/nu_max
    (the derivative of s nu(s) lies in [nu_min, 2 nu_max - nu_min])."""
    prob = W.unit_square_problem(9, 8, amps=(3000.0,))
    d = P.assemble(prob)
    res = P.fixed_point(prob, d, tol=1e-12, max_it=20000)
    assert res.converged
    U = res.U
    N = d.N
    assert np.abs(U[:, N // 2:] + U[:, :N // 2]).max() <= 1e-12 * np.abs(U).max()
    s = np.array(res.step_knorms)
    ratios = s[1:] / s[:-1]
    q = 1 - prob.nu_min / prob.nu_max
    assert ratios.max() <= q + 1e-9


def test_linear_rate_closed_form():
    """Linear material nu = c < nu_max on every element, zero source: the
    error propagator is P^{-1}(nu_max - c)A.  On the time-mean (k = 0) mode
    the periodic operator P reduces to nu_max A, so a time-constant start
    contracts by exactly 1 - c/nu_max per step; a start with zero time mean
    contracts strictly faster (Re of the discrete symbol > 0 for k != 0)."""
    c = 40.0
    prob = W.unit_square_problem(7, 4, amps=(0.0,))
    prob = prob.replace(nonlinear_e=np.zeros(prob.n_tri, np.uint8), nu_linear=c)
    d = P.assemble(prob)
    rng = np.random.default_rng(2)
    U0 = np.repeat(rng.normal(size=(d.n, 1)), d.N, axis=1)
    res = P.fixed_point(prob, d, U0=U0, tol=1e-8, max_it=60)
    s = np.array(res.step_knorms)
    np.testing.assert_allclose(s[1:] / s[:-1], 1 - c / prob.nu_max, rtol=1e-10)
    V0 = rng.normal(size=(d.n, d.N))
    V0 -= V0.mean(axis=1, keepdims=True)
    res = P.fixed_point(prob, d, U0=V0, tol=1e-8, max_it=60)
    s = np.array(res.step_knorms)
    assert (s[1:] / s[:-1]).max() < 1 - c / prob.nu_max - 1e-6


def test_zero_source_gives_zero():
    prob = W.unit_square_problem(7, 4, amps=(0.0,))
    res = P.fixed_point(prob, tol=1e-10, max_it=3)
    assert np.abs(res.U).max() == 0.0


def test_newton_jacobian_matches_differences():
    """The space-time Jacobian of A (used by Newton and the adjoint) is the
    derivative of A: J v = (A(U + h v) - A(U - h v)) / 2h."""
    prob = W.unit_square_problem(6, 4, amps=(2000.0,))
    d = P.assemble(prob)
    rng = np.random.default_rng(4)
    U = rng.normal(scale=0.05, size=(d.n, d.N))
    V = rng.normal(size=(d.n, d.N))
    J = P.jacobian(prob, d, U)
    h = 1e-7
    fd = (P.A_apply(prob, d, U + h * V) - P.A_apply(prob, d, U - h * V)) / (2 * h)
    np.testing.assert_allclose((J @ V.ravel()).reshape(V.shape), fd, rtol=1e-6, atol=1e-7)


# --------------------------------------------------------------------------
# Initialisation (Section 4): the decoupled static problems K(u^n) = f^n
# --------------------------------------------------------------------------

def test_static_solve_linear_material_is_a_linear_solve():
    """nu = c on every element makes K = c A, so the static problems are the
    linear systems c A u^n = f^n (a library sparse solve)."""
    c = 40.0
    prob = W.unit_square_problem(9, 6)
    prob = prob.replace(nonlinear_e=np.zeros(prob.n_tri, np.uint8), nu_linear=c)
    d = P.assemble(prob)
    F = P.source(prob, d)
    U, rel = P.static_solve(prob, d)
    ref = sp.linalg.spsolve((c * d.A).tocsc(), F)
    assert rel < 1e-14
    assert np.linalg.norm(U - ref) <= 1e-12 * np.linalg.norm(ref)


def test_static_solve_residual_zero_source_and_odd_symmetry():
    """A strongly saturated case reaches K(U) = F to rounding; K is odd, so
    -F gives -U; zero source gives U = 0."""
    prob = W.unit_square_problem(9, 4, amps=(4000.0,))
    d = P.assemble(prob)
    F = P.source(prob, d)
    U, rel = P.static_solve(prob, d)
    assert rel < 1e-13
    assert np.linalg.norm(F - P.K_free(prob, d, U)) <= 1e-12 * np.linalg.norm(F)
    full = P.lift(prob, d, U)
    s = np.sqrt((fem.element_gradients(prob, full) ** 2).sum(axis=1))
    iron = prob.nonlinear_e.astype(bool)
    assert s[iron].max() > prob.s_sat   # the iron saturates: nu is not constant
    Um, _ = P.static_solve(prob, d, F=-F)
    assert np.abs(Um + U).max() <= 1e-12 * np.abs(U).max()
    Z, _ = P.static_solve(prob, d, F=np.zeros_like(F))
    assert np.abs(Z).max() == 0.0


def test_static_solve_is_the_zero_conductivity_periodic_solution():
    """With sigma = 0 the mass term of Problem 1 vanishes and the time steps
    decouple: the periodic fixed point (exact inner solves) equals the static
    solutions.  The same holds for N = 1 with any sigma, since u^0 = u^1
    cancels the mass term."""
    prob = W.unit_square_problem(9, 4, amps=(3000.0,))
    prob0 = prob.replace(sigma_e=np.zeros(prob.n_tri))
    d0 = P.assemble(prob0)
    U, _ = P.static_solve(prob0, d0)
    res = P.fixed_point(prob0, d0, tol=1e-14, max_it=20000)
    assert res.converged
    assert np.linalg.norm(res.U - U) <= 1e-11 * np.linalg.norm(U)
    prob1 = W.unit_square_problem(9, 1, amps=(3000.0,))
    d1 = P.assemble(prob1)
    U1, _ = P.static_solve(prob1, d1)
    res1 = P.fixed_point(prob1, d1, tol=1e-14, max_it=20000)
    assert res1.converged
    assert np.linalg.norm(res1.U - U1) <= 1e-11 * np.linalg.norm(U1)


def test_static_jacobian_matches_differences():
    prob = W.unit_square_problem(6, 3, amps=(2000.0,))
    d = P.assemble(prob)
    rng = np.random.default_rng(8)
    U = rng.normal(scale=0.05, size=(d.n, d.N))
    V = rng.normal(size=(d.n, d.N))
    J = P.static_jacobian(prob, d, U)
    h = 1e-7
    fd = (P.K_free(prob, d, U + h * V) - P.K_free(prob, d, U - h * V)) / (2 * h)
    np.testing.assert_allclose((J @ V.ravel()).reshape(V.shape), fd, rtol=1e-6, atol=1e-7)


# --------------------------------------------------------------------------
# The paper's transformer (Section 4): exponential law, K_hat weights
# --------------------------------------------------------------------------

def test_exp_law_closed_forms():
    """nu = a min(exp(b s^2), c) + d: a + d at zero field, a c + d above the
    cap s^2 = ln(c)/b, continuous there; the paper's iron and steel constants
    make the saturated value the air value 1e7/(4 pi) to within 0.01%."""
    for key in ("iron", "steel"):
        _, a, b, c, d = W.PAPER_MATERIALS[key]
        assert fem.exp_law(0.0, a, b, c, d) == a + d
        xc = math.log(c) / b
        assert fem.exp_law(xc * (1 + 1e-12), a, b, c, d) == pytest.approx(a * c + d, rel=1e-10)
        assert fem.exp_law(xc * (1 - 1e-12), a, b, c, d) == pytest.approx(a * c + d, rel=1e-9)
        assert fem.exp_law(4 * xc, a, b, c, d) == a * c + d
        assert abs(a * c + d - W.PAPER_NU_AIR) < 1e-4 * W.PAPER_NU_AIR
        x = 0.3 * xc
        assert fem.exp_law(x, a, b, c, d) == pytest.approx(a * math.exp(b * x) + d, rel=1e-15)
        assert fem.dexp_law_ds2(x, a, b, c, d) == pytest.approx(a * b * math.exp(b * x), rel=1e-15)
        assert fem.dexp_law_ds2(2 * xc, a, b, c, d) == 0.0


def _paper_small(N=4, scale=1.0):
    prob = W.paper_transformer_problem(21, 27, N)
    return prob.replace(amp=prob.amp * scale)


def test_exp_law_K_is_gradient_of_coenergy_and_jacobian():
    """With the exponential law K(u) = grad E(u) and DK = d K / du, checked by
    central differences on a field that puts elements on both sides of the
    cap (s of a few tesla)."""
    prob = _paper_small()
    rng = np.random.default_rng(21)
    u = rng.normal(size=prob.n_nodes) * 0.04
    u[prob.dirichlet == 1] = 0.0
    g = fem.element_gradients(prob, u)
    s2 = (g * g).sum(axis=1)
    iron = prob.nonlinear_e.astype(bool)
    xc = np.log(prob.law_abcd[iron, 2]) / prob.law_abcd[iron, 1]
    assert (s2[iron] > xc).any() and (s2[iron] < xc).any()
    K = fem.K_apply(prob, u)
    v = rng.normal(size=prob.n_nodes)
    v[prob.dirichlet == 1] = 0.0
    h = 1e-9
    dE = (fem.energy(prob, u + h * v) - fem.energy(prob, u - h * v)) / (2 * h)
    assert dE == pytest.approx(float(K @ v), rel=1e-6)
    J = fem.K_jacobian(prob, u)
    fd = (fem.K_apply(prob, u + h * v) - fem.K_apply(prob, u - h * v)) / (2 * h)
    np.testing.assert_allclose(J @ v, fd, rtol=1e-5, atol=1e-6 * np.abs(fd).max())


def test_khat_weights_assemble_the_weighted_stiffness():
    """K_hat = sum_T khat_T A_T: a constant weight gives khat A; the weight of
    one right triangle with legs h gives its textbook element matrix
    [[1,-1,0],[-1,2,-1],[0,-1,1]]/2 (vertices in the order of the split)."""
    prob = _paper_small()
    free = prob.interior
    A = fem.restrict(fem.stiffness(prob.xy, prob.tri, np.ones(prob.n_tri)), free)
    L = P.assemble(prob.replace(khat_e=np.full(prob.n_tri, 7.5))).L
    assert abs(L - 7.5 * A).max() < 1e-12
    # element 0 = [(0,0), (1,0), (1,1)] of cell (0,0): legs h_x, h_y
    w = np.zeros(prob.n_tri)
    w[0] = 1.0
    Kel = fem.stiffness(prob.xy, prob.tri, w).toarray()
    hx = prob.xy[1, 0] - prob.xy[0, 0]
    hy = prob.xy[prob.grid[0], 1] - prob.xy[0, 1]
    t = prob.tri[0]
    ref = np.array([[hy / hx, -hy / hx, 0.0],
                    [-hy / hx, hy / hx + hx / hy, -hx / hy],
                    [0.0, -hx / hy, hx / hy]]) / 2.0
    np.testing.assert_allclose(Kel[np.ix_(t, t)], ref, rtol=1e-12, atol=1e-15)


def test_paper_transformer_fixed_point_matches_newton_and_linear_limit():
    """The fixed point with the zero-field K_hat weights reaches the unique
    solution found by the independent Newton solver; at a tiny current the
    problem is linear with nu = a + d on iron and steel."""
    prob = _paper_small()
    d = P.assemble(prob)
    Un, r = P.newton(prob, d, tol=1e-14)
    assert r < 1e-12
    res = P.fixed_point(prob, d, tol=1e-14, max_it=200)
    assert res.converged
    assert np.linalg.norm(res.U - Un) <= 1e-11 * np.linalg.norm(Un)
    small = _paper_small(scale=1e-6)
    ds = P.assemble(small)
    Us = P.fixed_point(small, ds, tol=1e-14, max_it=50).U
    # linear reference: K = K_hat (nu = a + d on iron and steel), one exact periodic solve
    ref = P.DFTSolver(ds.M, ds.L, ds.tau, ds.N).solve(P.source(small, ds))
    assert np.linalg.norm(Us - ref) <= 1e-9 * np.linalg.norm(ref)
