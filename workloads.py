"""Seeded synthetic problem data for the time-periodic eddy-current solver.

This module builds INPUTS only: structured P1 triangle meshes, per-element
materials (conductivity sigma, nonlinear flag), coil membership, coil
amplitudes and phases, the period T and the number of implicit-Euler steps N.
It holds none of the method's arithmetic (no gradients, areas, matrices,
residuals or solves), so that both the CPU oracle and the CUDA library can be
fed from it without sharing any computation.

The problem is the 2D magneto-quasistatic model of the paper's Section 4
(sigma d_t u - div(nu(|grad u|) grad u) = j, u = 0 on the boundary), on
synthetic geometries: a unit square with an iron block and strip coils, and a
transformer-shaped 2x1 rectangle with an iron frame and two window coils.

Material law (iron elements): nu(s) = nu_min + (nu_max - nu_min) s^2/(s^2 + s_sat^2),
or, when a problem carries per-element law constants `law_abcd` (the paper's
transformer, Section 4), nu(s) = a min(exp(b s^2), c) + d.  Non-iron elements
use the constant nu_linear.  The source in coil c is the element-constant
current density amp_c * sin(2 pi t / T + phase_c).  `khat_e`, when present,
gives per-element weights of the linear operator K_hat = sum_T khat_T A_T of
the fixed-point iteration (else K_hat = nu_max A).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Problem",
    "structured_mesh",
    "unit_square_problem",
    "transformer_problem",
    "config_plain_fp64",
    "config_mixed",
    "config_transformer",
    "config_adjoint",
    "config_batched",
    "one_node_problem",
    "delaunay_problem",
    "paper_transformer_problem",
    "config_paper_transformer",
]


@dataclasses.dataclass
class Problem:
    """One time-periodic problem instance (all arrays C-contiguous)."""

    name: str
    xy: np.ndarray            # (n_nodes, 2) float64 node coordinates
    tri: np.ndarray           # (n_tri, 3) int32 counter-clockwise vertex ids
    dirichlet: np.ndarray     # (n_nodes,) uint8, 1 = homogeneous Dirichlet node
    sigma_e: np.ndarray       # (n_tri,) float64 conductivity per element
    nonlinear_e: np.ndarray   # (n_tri,) uint8, 1 = iron (nonlinear nu law)
    coil_of_elem: np.ndarray  # (n_tri,) int32 coil index or -1
    amp: np.ndarray           # (n_coils,) float64 current-density amplitudes
    phase: np.ndarray         # (n_coils,) float64 phase shifts (radians)
    nu_min: float
    nu_max: float
    s_sat: float
    nu_linear: float
    T: float
    N: int
    grid: tuple | None = None  # (nx, ny, x0, y0, x1, y1) when structured
    law_abcd: np.ndarray | None = None  # (n_tri, 4) a, b, c, d of the exponential law, or None
    khat_e: np.ndarray | None = None    # (n_tri,) weights of K_hat, or None (nu_max everywhere)

    @property
    def n_nodes(self) -> int:
        return int(self.xy.shape[0])

    @property
    def n_tri(self) -> int:
        return int(self.tri.shape[0])

    @property
    def n_coils(self) -> int:
        return int(self.amp.shape[0])

    @property
    def interior(self) -> np.ndarray:
        """Indices of the free (non-Dirichlet) nodes in ascending order."""
        return np.flatnonzero(self.dirichlet == 0).astype(np.int64)

    @property
    def n_free(self) -> int:
        return int(np.count_nonzero(self.dirichlet == 0))

    def replace(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)


def structured_mesh(nx: int, ny: int, x0: float = 0.0, y0: float = 0.0,
                    x1: float = 1.0, y1: float = 1.0):
    """Uniform nx-by-ny node grid on [x0,x1]x[y0,y1].

    Node (i, j) has id j*nx + i.  Every cell is split along its diagonal from
    (i, j) to (i+1, j+1) into two counter-clockwise triangles
    [(i,j), (i+1,j), (i+1,j+1)] and [(i,j), (i+1,j+1), (i,j+1)].
    Boundary nodes are flagged Dirichlet.
    """
    if nx < 2 or ny < 2:
        raise ValueError("structured_mesh needs at least 2x2 nodes")
    xs = x0 + (x1 - x0) * np.arange(nx, dtype=np.float64) / (nx - 1)
    ys = y0 + (y1 - y0) * np.arange(ny, dtype=np.float64) / (ny - 1)
    X, Y = np.meshgrid(xs, ys)  # (ny, nx)
    xy = np.ascontiguousarray(np.stack([X.ravel(), Y.ravel()], axis=1))
    ii, jj = np.meshgrid(np.arange(nx - 1), np.arange(ny - 1))
    ii = ii.ravel()
    jj = jj.ravel()
    n00 = jj * nx + ii
    n10 = n00 + 1
    n11 = n00 + nx + 1
    n01 = n00 + nx
    lower = np.stack([n00, n10, n11], axis=1)
    upper = np.stack([n00, n11, n01], axis=1)
    # interleave lower/upper per cell so that element 2c, 2c+1 belong to cell c
    tri = np.empty((2 * lower.shape[0], 3), dtype=np.int32)
    tri[0::2] = lower
    tri[1::2] = upper
    dirichlet = np.zeros(nx * ny, dtype=np.uint8)
    b = np.zeros((ny, nx), dtype=bool)
    b[0, :] = b[-1, :] = b[:, 0] = b[:, -1] = True
    dirichlet[b.ravel()] = 1
    return xy, tri, dirichlet


def _centroids(xy, tri):
    # Region membership is decided by the triangle centroid (an input rule,
    # not part of the method).
    return xy[tri].mean(axis=1)


def _in_box(c, box):
    (a, b), (d, e) = box
    return (c[:, 0] > a) & (c[:, 0] < b) & (c[:, 1] > d) & (c[:, 1] < e)


def unit_square_problem(n: int, N: int, *, amps=(50.0,), phases=(0.0,),
                        coil_boxes=(((0.05, 0.2), (0.2, 0.8)),),
                        sigma_iron: float = 10.0, nu_min: float = 1.0,
                        nu_max: float = 100.0, s_sat: float = 1.0,
                        nu_linear: float = 100.0, T: float = 1.0,
                        sigma_sample: np.ndarray | None = None,
                        name: str | None = None) -> Problem:
    """Unit square, n x n nodes, iron block [0.25,0.75]^2, strip coil(s)."""
    xy, tri, dirichlet = structured_mesh(n, n)
    c = _centroids(xy, tri)
    iron = _in_box(c, ((0.25, 0.75), (0.25, 0.75)))
    coil = np.full(tri.shape[0], -1, dtype=np.int32)
    for k, box in enumerate(coil_boxes):
        coil[_in_box(c, box)] = k
    sigma = np.zeros(tri.shape[0], dtype=np.float64)
    if sigma_sample is not None:
        sigma[iron] = sigma_sample[: int(iron.sum())]
    else:
        sigma[iron] = sigma_iron
    return Problem(
        name=name or f"square{n}_N{N}", xy=xy, tri=tri, dirichlet=dirichlet,
        sigma_e=sigma, nonlinear_e=iron.astype(np.uint8), coil_of_elem=coil,
        amp=np.asarray(amps, dtype=np.float64),
        phase=np.asarray(phases, dtype=np.float64),
        nu_min=nu_min, nu_max=nu_max, s_sat=s_sat, nu_linear=nu_linear,
        T=T, N=int(N), grid=(n, n, 0.0, 0.0, 1.0, 1.0))


def transformer_problem(nx: int, ny: int, N: int, *, J0: float = 60.0,
                        sigma_iron: float = 5.0, T: float = 1.0,
                        name: str | None = None) -> Problem:
    """Transformer-shaped 2x1 rectangle: iron frame minus two windows, one
    coil inside each window with phases 0 and 2 pi/3."""
    xy, tri, dirichlet = structured_mesh(nx, ny, 0.0, 0.0, 2.0, 1.0)
    c = _centroids(xy, tri)
    frame = _in_box(c, ((0.25, 1.75), (0.125, 0.875)))
    w1 = _in_box(c, ((0.5, 0.875), (0.3125, 0.6875)))
    w2 = _in_box(c, ((1.125, 1.5), (0.3125, 0.6875)))
    iron = frame & ~w1 & ~w2
    coil = np.full(tri.shape[0], -1, dtype=np.int32)
    coil[_in_box(c, ((0.5625, 0.8125), (0.375, 0.625)))] = 0
    coil[_in_box(c, ((1.1875, 1.4375), (0.375, 0.625)))] = 1
    sigma = np.where(iron, sigma_iron, 0.0).astype(np.float64)
    return Problem(
        name=name or f"transformer{nx}x{ny}_N{N}", xy=xy, tri=tri,
        dirichlet=dirichlet, sigma_e=sigma, nonlinear_e=iron.astype(np.uint8),
        coil_of_elem=coil, amp=np.array([J0, J0]),
        phase=np.array([0.0, 2.0 * math.pi / 3.0]), nu_min=1.0, nu_max=100.0,
        s_sat=1.0, nu_linear=100.0, T=T, N=int(N),
        grid=(nx, ny, 0.0, 0.0, 2.0, 1.0))


def delaunay_problem(n_interior: int, N: int, seed: int = 0, *, amp: float = 50.0,
                     name: str | None = None) -> Problem:
    """Unstructured mesh of the unit square: Delaunay triangulation of
    `n_interior` seeded random points plus 12 points per side, with the iron
    block, a strip coil and the materials of the unit-square workloads
    (centroid rule).  Vertex degrees vary (some rows exceed 8 entries)."""
    from scipy.spatial import Delaunay
    rng = np.random.default_rng(seed)
    t = np.linspace(0.0, 1.0, 13)[:-1]
    side = [np.stack([t, np.zeros_like(t)], 1), np.stack([np.ones_like(t), t], 1),
            np.stack([1 - t, np.ones_like(t)], 1), np.stack([np.zeros_like(t), 1 - t], 1)]
    bnd = np.concatenate(side)
    pts = np.concatenate([bnd, 0.02 + 0.96 * rng.random((n_interior, 2))])
    tri = Delaunay(pts).simplices.astype(np.int32)
    p = pts[tri]
    det = (p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1]) - (p[:, 2, 0] - p[:, 0, 0]) * (p[:, 1, 1] - p[:, 0, 1])
    flip = det < 0
    tri[flip] = tri[flip][:, [0, 2, 1]]
    keep = np.abs(det) > 1e-12
    tri = np.ascontiguousarray(tri[keep])
    dirichlet = np.zeros(pts.shape[0], dtype=np.uint8)
    dirichlet[: bnd.shape[0]] = 1
    c = _centroids(pts, tri)
    iron = _in_box(c, ((0.25, 0.75), (0.25, 0.75)))
    coil = np.full(tri.shape[0], -1, dtype=np.int32)
    coil[_in_box(c, ((0.05, 0.2), (0.2, 0.8)))] = 0
    return Problem(
        name=name or f"delaunay{n_interior}_N{N}_seed{seed}", xy=np.ascontiguousarray(pts), tri=tri,
        dirichlet=dirichlet, sigma_e=np.where(iron, 10.0, 0.0), nonlinear_e=iron.astype(np.uint8),
        coil_of_elem=coil, amp=np.array([amp]), phase=np.array([0.0]), nu_min=1.0, nu_max=100.0,
        s_sat=1.0, nu_linear=100.0, T=1.0, N=int(N), grid=None)


def one_node_problem(N: int, *, sigma: float = 10.0, nonlinear: bool = True,
                     amp: float = 50.0, nu_min: float = 1.0,
                     nu_max: float = 100.0, s_sat: float = 1.0) -> Problem:
    """3x3 grid on the unit square: a single free node, every element iron
    (or linear) and a coil, so the discrete problem is scalar."""
    xy, tri, dirichlet = structured_mesh(3, 3)
    ne = tri.shape[0]
    return Problem(
        name=f"onenode_N{N}", xy=xy, tri=tri, dirichlet=dirichlet,
        sigma_e=np.full(ne, sigma), nonlinear_e=np.full(ne, 1 if nonlinear else 0, np.uint8),
        coil_of_elem=np.zeros(ne, np.int32), amp=np.array([amp]), phase=np.array([0.0]),
        nu_min=nu_min, nu_max=nu_max, s_sat=s_sat, nu_linear=nu_max, T=1.0,
        N=int(N), grid=(3, 3, 0.0, 0.0, 1.0, 1.0))


# ---------------------------------------------------------------------------
# The five named workloads
# ---------------------------------------------------------------------------

def config_plain_fp64() -> Problem:
    """33x33 nodes (2048 triangles), N = 32, J0 = 50, FP64, tol 1e-10."""
    return unit_square_problem(33, 32, name="square33_N32")


def config_mixed(seed: int = 0, n: int = 257, N: int = 256) -> Problem:
    """257x257 nodes (131072 triangles), N = 256, J0 ~ U[20, 80] from seed."""
    rng = np.random.default_rng(seed)
    J0 = float(rng.uniform(20.0, 80.0))
    return unit_square_problem(n, N, amps=(J0,), name=f"square{n}_N{N}_seed{seed}")


def config_transformer(nx: int = 1025, ny: int = 513, N: int = 512) -> Problem:
    """2x1 transformer-shaped rectangle, 1025x513 nodes, N = 512."""
    return transformer_problem(nx, ny, N)


def config_adjoint(seed: int = 0, n: int = 257, N: int = 256) -> Problem:
    """257x257, N = 256, two in-phase strip coils (amplitude 50 each) and a
    log-normal iron conductivity ln(sigma_e) ~ N(ln 10, 0.3^2)."""
    rng = np.random.default_rng(seed)
    n_tri = 2 * (n - 1) * (n - 1)
    sig = np.exp(rng.normal(math.log(10.0), 0.3, size=n_tri))
    return unit_square_problem(
        n, N, amps=(50.0, 50.0), phases=(0.0, 0.0),
        coil_boxes=(((0.05, 0.2), (0.2, 0.8)), ((0.8, 0.95), (0.2, 0.8))),
        sigma_sample=sig, name=f"adjoint{n}_N{N}_seed{seed}")


def config_batched(seed: int = 0, count: int = 64,
                   grids=(65, 129, 257, 513), steps=(64, 128, 256, 512)):
    """`count` independent instances with uneven mesh size and N."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        n = int(rng.choice(grids))
        N = int(rng.choice(steps))
        J0 = float(rng.uniform(20.0, 80.0))
        s_sat = float(rng.uniform(0.5, 2.0))
        out.append(unit_square_problem(n, N, amps=(J0,), s_sat=s_sat,
                                       name=f"batch{k}_n{n}_N{N}"))
    return out


# Section 4 of the paper: cross-section of a power transformer (figure of the
# domain and table of material constants), in metres.  Tank 355 x 466 mm with
# a 10 mm steel wall; iron core [60,295] x [28,438] mm minus the window
# [140,215] x [108,358] mm; four windings 13 x 220 mm with lower-left corners
# at x = 28, 159, 183, 314 mm, y = 123 mm (winding+ at 159 and 314, winding-
# at 28 and 183); air elsewhere.
PAPER_MATERIALS = {
    #         sigma [S/m], a [m/H], b, c, d [m/H]
    "iron": (0.0, 5.85, 2.196, 136026.0, 23.15),
    "steel": (1.0e7, 130.171, 1.102, 6112.97, 43.742),
}
PAPER_NU_AIR = 1.0e7 / (4.0 * math.pi)   # air and windings [m/H]
PAPER_J = 1.9e4                          # winding current density amplitude [A/m^2]
PAPER_T = 0.02                           # period [s]


def paper_transformer_problem(nx: int, ny: int, N: int, name: str | None = None) -> Problem:
    """The paper's transformer on a structured nx x ny node grid over the
    355 x 466 mm tank (regions by triangle centroid).  Iron and steel follow
    nu = a min(exp(b s^2), c) + d with the paper's constants; j = +-J cos(2 pi
    t / T) in the windings (phase pi/2 of the sine convention); T = 0.02 s.
    K_hat weights: the zero-field reluctivity of each element (a + d on iron
    and steel, the air value elsewhere)."""
    mm = 1.0e-3
    xy, tri, dirichlet = structured_mesh(nx, ny, 0.0, 0.0, 355 * mm, 466 * mm)
    c = _centroids(xy, tri)
    box = lambda x0, x1, y0, y1: _in_box(c, ((x0 * mm, x1 * mm), (y0 * mm, y1 * mm)))
    steel = ~box(10, 345, 10, 456)
    iron = box(60, 295, 28, 438) & ~box(140, 215, 108, 358)
    w_plus = box(159, 172, 123, 343) | box(314, 327, 123, 343)
    w_minus = box(28, 41, 123, 343) | box(183, 196, 123, 343)
    coil = np.full(tri.shape[0], -1, dtype=np.int32)
    coil[w_plus] = 0
    coil[w_minus] = 1
    n_tri = tri.shape[0]
    sigma = np.zeros(n_tri)
    abcd = np.zeros((n_tri, 4))
    for mask, key in ((iron, "iron"), (steel, "steel")):
        sg, a, b, cc, d = PAPER_MATERIALS[key]
        sigma[mask] = sg
        abcd[mask] = (a, b, cc, d)
    nonlinear = (iron | steel).astype(np.uint8)
    khat = np.where(nonlinear == 1, abcd[:, 0] + abcd[:, 3], PAPER_NU_AIR)
    return Problem(
        name=name or f"paper_transformer{nx}x{ny}_N{N}", xy=xy, tri=tri, dirichlet=dirichlet,
        sigma_e=sigma, nonlinear_e=nonlinear, coil_of_elem=coil,
        amp=np.array([PAPER_J, -PAPER_J]), phase=np.array([0.5 * math.pi, 0.5 * math.pi]),
        nu_min=1.0, nu_max=1.0, s_sat=1.0, nu_linear=PAPER_NU_AIR, T=PAPER_T, N=int(N),
        grid=(nx, ny, 0.0, 0.0, 355 * mm, 466 * mm), law_abcd=abcd, khat_e=khat)


def config_paper_transformer(size: str = "8208", N: int = 128) -> Problem:
    """The paper's transformer at its two mesh sizes, matched approximately by
    structured grids: N_V = 8208 -> 81 x 105 nodes (8137 free), N_V = 32451 ->
    161 x 209 nodes (32913 free); N in {128, 256, 512}."""
    nx, ny = {"8208": (81, 105), "32451": (161, 209)}[size]
    return paper_transformer_problem(nx, ny, N, name=f"paper_transformer{size}_N{N}")
