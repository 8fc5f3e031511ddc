"""The structured-grid stencil kernels of the float inner solve against the
padded-ELL row kernels they replace, and the solves that use them against the
oracle.

The stencil path reorders float sums (a 7-point stencil instead of an ELL row,
fused passes), so one multigrid-in-time cycle agrees with the ELL path to
float rounding (relative 1e-5 here), and the converged fixed points both reach
the oracle's solution at the mixed-precision bar 1e-8.  Cases: the bench
grid's hierarchy on small grids, odd step counts (time levels with 3 steps,
one float per thread), two steps, and a rectangle."""
import os

import numpy as np
import pytest

import workloads as W
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


# (name, problem, extra options): N = 12 and N = 6 stop at a 3-step level,
# solved exactly by the DFT in time; their float levels have 12 and 6 steps
# (6 columns: three threads per node, 85 nodes per block)
CASES = [
    ("square33_N32", lambda: W.unit_square_problem(33, 32), {}),
    ("square65_N12", lambda: W.unit_square_problem(65, 12, amps=(70.0,)), {"coarse_solver": 1}),
    ("square17_N6", lambda: W.unit_square_problem(17, 6), {"coarse_solver": 1}),
    ("square17_N2", lambda: W.unit_square_problem(17, 2), {}),
    ("transformer65x33_N16", lambda: W.transformer_problem(65, 33, 16), {}),
]


@pytest.mark.parametrize("name,make,extra", CASES, ids=[c[0] for c in CASES])
def test_one_cycle_matches_the_ell_kernels(name, make, extra):
    prob = make()
    n, N = prob.n_free, prob.N
    rng = np.random.default_rng(4)
    B = torch.tensor(rng.normal(size=(n, N)), device="cuda")
    out = []
    for stencil in (0, 1):
        c, o = _ctx(prob, precision=ptp.PTP_MIXED, stencil=stencil, **extra)
        X = torch.empty_like(B)
        rel = c.periodic_solve_dev(B, X, 1, o)
        out.append((X.cpu().numpy(), rel))
    (x0, r0), (x1, r1) = out
    assert np.linalg.norm(x1 - x0) <= 1e-5 * np.linalg.norm(x0)
    assert abs(r1 - r0) <= 1e-4 * max(r0, 1e-30) + 1e-6
    assert r1 < 0.5          # one cycle reduces the residual


# fixed points against the oracle (exact inner solves, to 1e-13); the 33x33,
# N = 32 solution is the stored one of tests/golden
ORACLE_CASES = [
    ("square33_N32", lambda: W.unit_square_problem(33, 32), {}),
    ("square33_N12", lambda: W.unit_square_problem(33, 12, amps=(70.0,)), {"coarse_solver": 1}),
    ("square17_N6", lambda: W.unit_square_problem(17, 6), {"coarse_solver": 1}),
    ("square17_N2", lambda: W.unit_square_problem(17, 2), {}),
    ("transformer33x17_N16", lambda: W.transformer_problem(33, 17, 16), {}),
]


@pytest.mark.parametrize("name,make,extra", ORACLE_CASES, ids=[c[0] for c in ORACLE_CASES])
def test_fixed_point_with_stencil_kernels_reaches_the_oracle(name, make, extra):
    prob = make()
    if name == "square33_N32":
        Uo = np.load(os.path.join(GOLDEN, "square33_N32_oracle.npz"))["U"]
    else:
        d = P.assemble(prob)
        ref = P.fixed_point(prob, d, tol=1e-13, max_it=50000)
        assert ref.converged
        Uo = ref.U
    its = []
    for stencil in (1, 0):
        c, o = _ctx(prob, precision=ptp.PTP_MIXED, stencil=stencil, tol=1e-11, max_outer=20000, **extra)
        U, st, rc = c.solve(o)
        assert rc == ptp.PTP_OK
        err = np.linalg.norm(U - Uo) / np.linalg.norm(Uo)
        assert err < 1e-8, (stencil, err)
        its.append(st.outer_iterations)
    # the same iteration up to float rounding: outer counts within a few steps
    assert abs(its[0] - its[1]) <= max(3, its[1] // 100), its


def test_stencil_path_launches_fewer_kernels():
    prob = W.unit_square_problem(65, 32)
    counts = []
    for stencil in (0, 1):
        c, o = _ctx(prob, precision=ptp.PTP_MIXED, stencil=stencil, tol=1e-8, max_outer=3)
        U = torch.zeros((prob.n_free, prob.N), dtype=torch.float64, device="cuda")
        st, rc = c.solve_dev(U, o)
        counts.append(st.kernel_launches / max(1, st.outer_iterations + 1))
    assert counts[1] < 0.8 * counts[0], counts


@pytest.mark.parametrize("precision,tol,bar", [(ptp.PTP_FP64, 1e-13, 1e-10), (ptp.PTP_MIXED, 1e-11, 1e-8)])
def test_fixed_point_with_the_fused_residual_reaches_the_oracle(precision, tol, bar):
    """The one-pass structured outer residual (k1_fused) inside the fixed
    point: the 33x33, N = 32 solve reaches the stored oracle solution."""
    prob = W.unit_square_problem(33, 32)
    Uo = np.load(os.path.join(GOLDEN, "square33_N32_oracle.npz"))["U"]
    c, o = _ctx(prob, precision=precision, tol=tol, max_outer=20000, k1_fused=1)
    U, st, rc = c.solve(o)
    assert rc == ptp.PTP_OK
    assert np.linalg.norm(U - Uo) / np.linalg.norm(Uo) < bar


@pytest.mark.parametrize("name,make", [("square33_N32", lambda: W.unit_square_problem(33, 32)),
                                       ("square17_N6", lambda: W.unit_square_problem(17, 6)),
                                       ("transformer65x33_N16", lambda: W.transformer_problem(65, 33, 16))])
def test_periodic_residual_f32_against_the_oracle(name, make):
    """ptp_periodic_residual_f32_dev at every time level: B - [(M + tau_l L)
    X^n - M X^{n-1}] in float against the oracle's double operator, to float
    rounding of the seven-point sums: 1e-5 of |B| + |M + tau_l L| |X^n| +
    |M| |X^{n-1}| elementwise (float rounding alone gives about 3e-7)."""
    prob = make()
    d = P.assemble(prob)
    c, o = _ctx(prob, precision=ptp.PTP_MIXED)
    rng = np.random.default_rng(11)
    levels = c.sizes()[3]
    for l in range(levels):
        Nl = prob.N >> l
        if Nl < 1 or prob.N % (1 << l):
            break
        tau = d.tau * (1 << l)
        X = rng.normal(size=(d.n, Nl))
        B = rng.normal(size=(d.n, Nl))
        PX = (d.M + tau * d.L) @ X - d.M @ np.roll(X, 1, axis=1)
        ref = B - PX
        Xd = torch.tensor(X, dtype=torch.float32, device="cuda")
        Bd = torch.tensor(B, dtype=torch.float32, device="cuda")
        Rd = torch.empty_like(Xd)
        c.periodic_residual_f32_dev(l, Xd, Bd, Rd)
        scale = np.abs(B) + abs(d.M + tau * d.L) @ np.abs(X) + abs(d.M) @ np.abs(np.roll(X, 1, axis=1))
        err = np.abs(Rd.cpu().numpy() - ref)
        assert np.all(err <= 1e-5 * scale + 1e-30), (l, float((err / scale).max()))


@pytest.mark.parametrize("name,make", [("square33_N32", lambda: W.unit_square_problem(33, 32)),
                                       ("square65_N64", lambda: W.unit_square_problem(65, 64, amps=(70.0,))),
                                       ("transformer65x33_N16", lambda: W.transformer_problem(65, 33, 16))])
def test_fused_coarse_levels_are_bitwise_the_separate_launches(name, make):
    """With fuse_coarse = 1 the time levels with at most 16 steps run as one
    cooperative kernel: every virtual block computes what the block of the
    separate launch computed, so the fixed point's iterates and iteration
    counts are identical, and the fused step issues fewer launches."""
    prob = make()
    out = []
    for fuse in (0, 1):
        c, o = _ctx(prob, precision=ptp.PTP_MIXED, tol=1e-10, max_outer=20000, fuse_coarse=fuse)
        U = torch.zeros((prob.n_free, prob.N), dtype=torch.float64, device="cuda")
        st, rc = c.solve_dev(U, o)
        assert rc == ptp.PTP_OK
        out.append((U.cpu().numpy(), st.outer_iterations, st.kernel_launches / (st.outer_iterations + 1)))
    (u0, i0, l0), (u1, i1, l1) = out
    assert i0 == i1
    assert np.array_equal(u0, u1)
    assert l1 < l0


@pytest.mark.parametrize("name,make,extra", [
    ("square33_N32", lambda: W.unit_square_problem(33, 32), {}),
    ("square65_N12", lambda: W.unit_square_problem(65, 12, amps=(70.0,)), {"coarse_solver": 1}),
    ("transformer65x33_N16", lambda: W.transformer_problem(65, 33, 16), {}),
    ("square33_N32_fused", lambda: W.unit_square_problem(33, 32), {"fuse_coarse": 1}),
    ("square33_N32_fp64", lambda: W.unit_square_problem(33, 32), {"precision": ptp.PTP_FP64, "tol": 1e-11}),
])
def test_update_handed_to_the_restriction_is_bitwise_the_update_kernel(name, make, extra):
    """With fuse_update = 1 (default) the pre-sweep from zero leaves
    x = omega_t alpha p to the time restriction, which forms and stores it
    (the same float products as the update kernel), and the prolongations of
    the V(1, 0) cycle and the update of U run as one pass summing the levels
    from the coarsest in the order of the level-by-level prolongations: the
    iterates and iteration counts are identical, with fewer launches."""
    prob = make()
    out = []
    for fuse in (0, 1):
        kw = dict(precision=ptp.PTP_MIXED, tol=1e-10, max_outer=20000)
        kw.update(extra)
        c, o = _ctx(prob, fuse_update=fuse, **kw)
        U = torch.zeros((prob.n_free, prob.N), dtype=torch.float64, device="cuda")
        st, rc = c.solve_dev(U, o)
        assert rc == ptp.PTP_OK
        out.append((U.cpu().numpy(), st.outer_iterations, st.kernel_launches / (st.outer_iterations + 1)))
    (u0, i0, l0), (u1, i1, l1) = out
    assert i0 == i1
    assert np.array_equal(u0, u1)
    assert l1 < l0


def test_shared_memory_limit_never_shrinks_in_a_fresh_process():
    """The same stencil kernel is launched from several call sites with ring
    sizes that differ per time level (the restriction after a sweep from
    zero, and after a sweep from a nonzero iterate).  Its dynamic
    shared-memory limit must only grow: a fresh process (nothing granted
    yet) running a few mixed multigrid-in-time cycles, whose first cycle
    takes one call site and later cycles the other, completes."""
    import subprocess
    import sys
    script = (
        "import sys; sys.path.insert(0, '.'); import numpy as np, torch, workloads as W\n"
        "from paper_2502_21013_gb300 import ptp\n"
        "p = W.config_plain_fp64(); c = ptp.Context(0); ptp.load_problem(c, p)\n"
        "o = ptp.default_opts(precision=ptp.PTP_MIXED); c.setup(o)\n"
        "n, N, _, _ = c.sizes()\n"
        "B = torch.tensor(np.random.default_rng(4).normal(size=(n, N)), device='cuda')\n"
        "X = torch.empty_like(B)\n"
        "r = c.periodic_solve_dev(B, X, 8, o)\n"
        "assert r < 1e-3, r\n"
        "print('ok')\n")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "-c", script], cwd=root, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0 and "ok" in out.stdout, out.stdout[-2000:] + out.stderr[-2000:]
