"""Captured graphs and buffer reallocation.

An outer step is captured once as a CUDA graph and replayed by later solves.
Entry points that need larger work buffers (the periodic solve's staging,
the adjoint and Newton work) reallocate them after such a capture; the graph
must then be captured again rather than replay the old addresses.  Each case
checks that a solve after the reallocation returns exactly the first
solve's iterate."""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
ptp = pytest.importorskip("paper_2502_21013_gb300.ptp")


@pytest.mark.parametrize("precision", [ptp.PTP_MIXED, ptp.PTP_FP64])
def test_solve_after_entry_points_that_grow_buffers(precision):
    prob = W.unit_square_problem(17, 8, amps=(2000.0,))
    c = ptp.Context(0)
    ptp.load_problem(c, prob)
    o = ptp.default_opts(precision=precision, tol=1e-10, max_outer=20000)
    c.setup(o)
    U1, st1, rc1 = c.solve(o)
    assert rc1 == ptp.PTP_OK
    n, N = prob.n_free, prob.N
    B = torch.randn((n, N), dtype=torch.float64, device="cuda")
    X = torch.empty_like(B)
    c.periodic_solve_dev(B, X, 2, o)          # grows the staging buffers
    U2, st2, rc2 = c.solve(o)
    assert rc2 == ptp.PTP_OK and st2.outer_iterations == st1.outer_iterations
    assert np.array_equal(U1, U2)
    Ud = torch.tensor(U1, device="cuda")
    c.adjoint_gradient_dev(Ud, o)             # allocates the adjoint work
    U3, _, _ = c.solve(o)
    assert np.array_equal(U1, U3)
    c.newton_solve(ptp.default_opts(precision=precision, tol=1e-8, max_outer=20))
    U4, _, _ = c.solve(o)
    assert np.array_equal(U1, U4)
