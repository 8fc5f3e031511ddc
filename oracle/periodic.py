"""Discrete time-periodic problem, its exact linear solvers and the fixed point.

Problem 1 (eq. disc1-disc2): find U = (u^1..u^N) with
    M d_tau u^n + K(u^n) = f^n,  n = 1..N,   u^0 = u^N,
where d_tau u^n = (u^n - u^{n-1}) / tau, tau = T/N, t^n = n tau.

Storage convention of this module (and of the CUDA library's interface):
U is an (n_V, N) array over the free nodes in ascending node id, column
n-1 holding u^n.  The periodic closure u^0 = u^N makes the previous step of
column 0 the last column, i.e. u^{n-1} is np.roll(U, 1, axis=1).

The fixed-point iteration of eq. (iter1)-(iter2) with a linear symmetric
elliptic K_hat = L = nu_max * A (stiffness with unit coefficient) needs in
every step the solution of the periodic, time-invariant linear system
    M d_tau x^n + L x^n = b^n,  x^0 = x^N.
It is solved EXACTLY here, either by a sparse LU factorisation of the full
space-time matrix or, following the Remark on parallel solvers (Section 3),
by a discrete Fourier transform in time that block-diagonalises it.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import fem


@dataclasses.dataclass
class Disc:
    """Assembled operators restricted to the free nodes."""
    free: np.ndarray      # free node ids (ascending)
    M: sp.csr_matrix      # sigma-weighted consistent mass
    A: sp.csr_matrix      # stiffness with unit coefficient
    L: sp.csr_matrix      # K_hat = nu_max * A, or sum_T khat_T A_T
    b: np.ndarray         # (n_coils, n_V) coil load vectors
    tau: float
    N: int

    @property
    def n(self) -> int:
        return int(self.free.shape[0])


def assemble(prob) -> Disc:
    """Section 4 "Simulation setup": P1 in space, implicit Euler with tau = T/N."""
    free = prob.interior
    ones = np.ones(prob.n_tri)
    A = fem.restrict(fem.stiffness(prob.xy, prob.tri, ones), free)
    M = fem.restrict(fem.mass(prob.xy, prob.tri, prob.sigma_e), free)
    b = fem.coil_load(prob)[:, free]
    if prob.khat_e is not None:   # K_hat = sum_T khat_T A_T (element weights of the problem)
        L = fem.restrict(fem.stiffness(prob.xy, prob.tri, prob.khat_e), free)
    else:
        L = (prob.nu_max * A).tocsr()
    return Disc(free=free, M=M, A=A, L=L, b=b, tau=prob.T / prob.N, N=prob.N)


def lift(prob, disc, U):
    """Zero extension of free-node vectors (n_V, ...) to all nodes."""
    full = np.zeros((prob.n_nodes,) + U.shape[1:])
    full[disc.free] = U
    return full


def K_free(prob, disc, U):
    """K(u^n) on the free nodes for every column of U (n_V, N)."""
    return fem.K_apply(prob, lift(prob, disc, U))[disc.free]


def source(prob, disc):
    """F = (f^1..f^N):  f^n = sum_c amp_c sin(2 pi t^n / T + phase_c) b_c,
    sampled at t^n = n tau (Problem 1 takes f^n as given; the current density
    is element-constant on each coil, Section 4)."""
    t = disc.tau * np.arange(1, disc.N + 1)
    s = np.sin(2.0 * math.pi * t[None, :] / prob.T + prob.phase[:, None])  # (n_coils, N)
    return (prob.amp[:, None, None] * s[:, None, :] * disc.b[:, :, None]).sum(axis=0)


def A_apply(prob, disc, U):
    """A(U)^n = M d_tau u^n + K(u^n) with u^0 = u^N (proof of Theorem 2)."""
    dU = (U - np.roll(U, 1, axis=1)) / disc.tau
    return disc.M @ dU + K_free(prob, disc, U)


def residual(prob, disc, U, F=None):
    """F - A(U), the finite element residual used in the stopping rule."""
    if F is None:
        F = source(prob, disc)
    return F - A_apply(prob, disc, U)


def knorm(disc, U):
    """||U||_{K_hat} = sqrt(sum_n <L u^n, u^n>)  (Theorem 3)."""
    return math.sqrt(float(np.sum(U * (disc.L @ U))))


# ---------------------------------------------------------------------------
# Exact solvers of the periodic time-invariant linear system
#     M (x^n - x^{n-1}) / tau + Khat x^n = b^n,   x^0 = x^N
# ---------------------------------------------------------------------------

def periodic_matrix(M, Khat, tau, N):
    """The space-time matrix in the (n_V, N) C-order layout (index i*N + n):
    kron(M/tau + Khat, I_N) - kron(M/tau, S) with the cyclic shift S."""
    S = sp.csr_matrix((np.ones(N), (np.arange(N), (np.arange(N) - 1) % N)), shape=(N, N))
    I = sp.identity(N, format="csr")
    return (sp.kron(M / tau + Khat, I) - sp.kron(M / tau, S)).tocsc()


class SpaceTimeLU:
    """Sparse LU of the full space-time matrix (tiny sizes only)."""

    def __init__(self, M, Khat, tau, N):
        self.N = N
        self.lu = spla.splu(periodic_matrix(M, Khat, tau, N))

    def solve(self, B):
        return self.lu.solve(np.ascontiguousarray(B).ravel()).reshape(B.shape)


class DFTSolver:
    """Time-DFT block diagonalisation (Remark on parallel solvers, Section 3).

    With X_k = sum_n x^n exp(-2 pi i k n / N), the cyclic backward difference
    becomes multiplication by (1 - exp(-2 pi i k/N)) / tau, so each mode solves
        ((1 - exp(-2 pi i k/N))/tau M + Khat) X_k = B_k.
    (The continuous-time symbol i omega_k of the Remark is replaced by this
    discrete one.)  Real data: modes k = 0..N/2 suffice (rfft).
    """

    def __init__(self, M, Khat, tau, N, keep_factors=True):
        self.M, self.Khat, self.tau, self.N = M.tocsc(), Khat.tocsc(), tau, N
        self.keep = keep_factors
        self.lus = {}

    def symbol(self, k):
        return (1.0 - np.exp(-2j * math.pi * k / self.N)) / self.tau

    def _factor(self, k):
        lam = self.symbol(k)
        if abs(lam.imag) < 1e-300:
            mat = (lam.real * self.M + self.Khat).tocsc()
        else:
            mat = (lam * self.M.astype(np.complex128) + self.Khat.astype(np.complex128)).tocsc()
        return spla.splu(mat)

    def solve(self, B):
        Bh = np.fft.rfft(B, axis=1)
        Xh = np.empty_like(Bh)
        for k in range(Bh.shape[1]):
            lu = self.lus.get(k)
            if lu is None:
                lu = self._factor(k)
                if self.keep:
                    self.lus[k] = lu
            rhs = Bh[:, k]
            if np.iscomplexobj(lu.L.data) or lu.L.dtype.kind == "c":
                Xh[:, k] = lu.solve(rhs.astype(np.complex128))
            else:
                Xh[:, k] = lu.solve(rhs.real) + 1j * lu.solve(rhs.imag)
        return np.fft.irfft(Xh, n=self.N, axis=1)


def dense_periodic_solve(M, Khat, tau, B):
    """Brute force: dense solve of the full space-time system (tiny only)."""
    P = periodic_matrix(M, Khat, tau, B.shape[1]).toarray()
    return np.linalg.solve(P, B.ravel()).reshape(B.shape)


# ---------------------------------------------------------------------------
# Fixed-point iteration, eq. (iter1)-(iter2)
# ---------------------------------------------------------------------------

@dataclasses.dataclass
class FixedPointResult:
    U: np.ndarray
    iterations: int
    res_history: list          # ||F - A(U^k)||_l2 for k = 0..iterations
    step_knorms: list          # ||U^{k+1} - U^k||_{K_hat}
    converged: bool


def fixed_point(prob, disc=None, U0=None, tol=1e-10, max_it=10000,
                inner="dft", Khat=None, F=None, solver=None):
    """Fixed-point iteration of eq. (iter1)-(iter2):
        M d_tau u^{n,k+1} + Khat u^{n,k+1} = f^n + Khat u^{n,k} - K(u^{n,k}),
        u^{0,k+1} = u^{N,k+1},
    each step solved exactly; stopped when ||F - A(U^k)|| <= tol ||F - A(U^0)||
    (stopping rule of Section 4, "Initialization")."""
    if disc is None:
        disc = assemble(prob)
    Khat = disc.L if Khat is None else Khat
    if F is None:
        F = source(prob, disc)
    if solver is None:
        solver = (DFTSolver(disc.M, Khat, disc.tau, disc.N) if inner == "dft"
                  else SpaceTimeLU(disc.M, Khat, disc.tau, disc.N))
    U = np.zeros((disc.n, disc.N)) if U0 is None else np.array(U0, dtype=np.float64)
    r0 = float(np.linalg.norm(residual(prob, disc, U, F)))
    hist = [r0]
    steps = []
    converged = r0 == 0.0
    k = 0
    while not converged and k < max_it:
        rhs = F + Khat @ U - K_free(prob, disc, U)
        U_new = solver.solve(rhs)
        steps.append(knorm(disc, U_new - U))
        U = U_new
        k += 1
        r = float(np.linalg.norm(residual(prob, disc, U, F)))
        hist.append(r)
        converged = r <= tol * r0
    return FixedPointResult(U=U, iterations=k, res_history=hist,
                            step_knorms=steps, converged=converged)


# ---------------------------------------------------------------------------
# Initialisation (Section 4): the decoupled nonlinear static problems
# ---------------------------------------------------------------------------

def static_jacobian(prob, disc, U):
    """Block-diagonal Jacobian of U -> (K(u^1)..K(u^N)) in the (n_V, N) C-order
    layout: block n is DK(u^n) restricted to the free nodes."""
    n, N = U.shape
    full = lift(prob, disc, U)
    rows, cols, vals = [], [], []
    for j in range(N):
        D = fem.restrict(fem.K_jacobian(prob, full[:, j]), disc.free).tocoo()
        rows.append(D.row * N + j); cols.append(D.col * N + j); vals.append(D.data)
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n * N, n * N))


def static_solve(prob, disc=None, tol=1e-14, max_it=60, F=None):
    """The initialisation of Section 4: with sigma = 0 the mass term drops and
    the time steps decouple into the nonlinear static problems
        K(u^n) = f^n,   n = 1..N.
    Solved here by Newton with step halving on ||F - K(U)|| (all N problems
    at once through the block-diagonal Jacobian, sparse direct solves), from
    U = 0, until ||F - K(U)|| <= tol ||F||."""
    if disc is None:
        disc = assemble(prob)
    if F is None:
        F = source(prob, disc)
    U = np.zeros((disc.n, disc.N))
    R = F - K_free(prob, disc, U)
    r0 = float(np.linalg.norm(R))
    r = r0
    for _ in range(max_it):
        if r <= tol * max(r0, 1e-300):
            break
        J = static_jacobian(prob, disc, U).tocsc()
        dU = spla.spsolve(J, R.ravel()).reshape(U.shape)
        t = 1.0
        while True:
            Un = U + t * dU
            Rn = F - K_free(prob, disc, Un)
            rn = float(np.linalg.norm(Rn))
            if rn < r or t < 1e-4:
                break
            t *= 0.5
        U, R, r = Un, Rn, rn
    return U, r / max(r0, 1e-300)


# ---------------------------------------------------------------------------
# Independent brute force: Newton on A(U) = F (tiny meshes)
# ---------------------------------------------------------------------------

def jacobian(prob, disc, U):
    """Jacobian of A at U in the (n_V, N) C-order layout: diagonal blocks
    M/tau + DK(u^n), cyclic sub-diagonal blocks -M/tau."""
    n, N = U.shape
    full = lift(prob, disc, U)
    rows, cols, vals = [], [], []
    Mt = (disc.M / disc.tau).tocoo()
    for j in range(N):
        D = fem.restrict(fem.K_jacobian(prob, full[:, j]), disc.free).tocoo()
        blk = (D + Mt).tocoo()
        rows.append(blk.row * N + j); cols.append(blk.col * N + j); vals.append(blk.data)
        jm = (j - 1) % N
        rows.append(Mt.row * N + j); cols.append(Mt.col * N + jm); vals.append(-Mt.data)
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n * N, n * N))


def newton(prob, disc=None, U0=None, tol=1e-14, max_it=50, F=None):
    """Plain Newton with step halving on ||F - A(U)||; sparse direct solves."""
    if disc is None:
        disc = assemble(prob)
    if F is None:
        F = source(prob, disc)
    U = np.zeros((disc.n, disc.N)) if U0 is None else np.array(U0, dtype=np.float64)
    R = residual(prob, disc, U, F)
    r0 = float(np.linalg.norm(R))
    r = r0
    for _ in range(max_it):
        if r <= tol * max(r0, 1e-300):
            break
        J = jacobian(prob, disc, U).tocsc()
        dU = spla.spsolve(J, R.ravel()).reshape(U.shape)
        t = 1.0
        while True:
            Un = U + t * dU
            Rn = residual(prob, disc, Un, F)
            rn = float(np.linalg.norm(Rn))
            if rn < r or t < 1e-4:
                break
            t *= 0.5
        U, R, r = Un, Rn, rn
    return U, r / max(r0, 1e-300)
