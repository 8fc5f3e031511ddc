"""Newton's method (method (M2) of Section 4) on the GPU against the oracle.

The Jacobian J = dA/dU (blocks M/tau + DK(u^n), cyclic -M/tau) applied by the
library is compared with the oracle's assembled space-time Jacobian; the
Newton iterate with the oracle's solution of Problem 1 (unique, Theorem 2).
Tolerances: Jacobian apply 1e-13; converged solutions 1e-10 (FP64) and 1e-8
(mixed), as in the other parity tests.
"""
import os

import numpy as np
import pytest

import workloads as W
from oracle import periodic as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
ptp = pytest.importorskip("paper_2502_21013_gb300.ptp")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(b), 1e-300))


def make_ctx(prob, structured=True, **opts):
    c = ptp.Context(0)
    ptp.load_problem(c, prob, structured=structured)
    o = ptp.default_opts(**opts)
    c.setup(o)
    return c, o


def cuda(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("structured", [True, False])
def test_jacobian_apply_matches_the_assembled_jacobian(structured):
    prob = W.unit_square_problem(17, 6, amps=(2000.0,))
    d = P.assemble(prob)
    c, _ = make_ctx(prob, structured, precision=ptp.PTP_FP64)
    rng = np.random.default_rng(9)
    for scale in (1e-3, 0.5):   # nearly linear and strongly saturated iron
        U = rng.normal(scale=scale, size=(d.n, d.N))
        V = rng.normal(size=(d.n, d.N))
        Y = torch.empty((d.n, d.N), dtype=torch.float64, device="cuda")
        c.jacobian_apply_dev(cuda(U), cuda(V), Y)
        ref = (P.jacobian(prob, d, U) @ V.ravel()).reshape(V.shape)
        assert rel(Y.cpu().numpy(), ref) < 1e-13


@pytest.mark.parametrize("precision,tol,bar", [("fp64", 1e-13, 1e-10), ("mixed", 1e-11, 1e-8)])
def test_newton_against_stored_oracle(precision, tol, bar):
    """config square33_N32: Newton reaches the oracle's fixed point in far
    fewer outer steps than the fixed-point iteration."""
    prob = W.config_plain_fp64()
    Uo = np.load(os.path.join(GOLDEN, "square33_N32_oracle.npz"))["U"]
    prec = ptp.PTP_FP64 if precision == "fp64" else ptp.PTP_MIXED
    c, o = make_ctx(prob, precision=prec, tol=tol, max_outer=40)
    U, st, rc = c.newton_solve(o)
    assert rc == ptp.PTP_OK and st.converged
    assert st.outer_iterations <= 25 and st.inner_iterations > 0
    assert rel(U, Uo) < bar


@pytest.mark.parametrize("precision,tol,bar", [("fp64", 1e-13, 1e-10), ("mixed", 1e-11, 1e-8)])
def test_newton_strongly_saturated_with_static_start(precision, tol, bar):
    prob = W.unit_square_problem(17, 16, amps=(3000.0,))
    d = P.assemble(prob)
    ref = P.fixed_point(prob, d, tol=1e-13, max_it=50000)
    assert ref.converged
    prec = ptp.PTP_FP64 if precision == "fp64" else ptp.PTP_MIXED
    for init in (0, 1):
        # from the static start the first residual is smaller than ||F||, so the
        # relative tolerance is capped above the double rounding floor
        c, o = make_ctx(prob, precision=prec, tol=max(tol, 1e-12) if init else tol, max_outer=40,
                        init_static=init, init_tol=1e-10)
        U, st, rc = c.newton_solve(o)
        assert rc == ptp.PTP_OK
        assert (st.init_iterations > 0) == bool(init)
        assert rel(U, ref.U) < bar
        Ud = torch.empty((d.n, d.N), dtype=torch.float64, device="cuda")
        st2, rc2 = c.newton_solve_dev(Ud, o)
        assert rc2 == ptp.PTP_OK and np.array_equal(Ud.cpu().numpy(), U)


def test_newton_rejects_unsupported_cases():
    prob = W.paper_transformer_problem(21, 27, 4)
    c, o = make_ctx(prob, precision=ptp.PTP_FP64, tol=1e-8, max_outer=5)
    with pytest.raises(ptp.PtpError):
        c.newton_solve(o)
    prob2 = W.unit_square_problem(9, 4)
    c2, o2 = make_ctx(prob2, precision=ptp.PTP_FP64, tol=1e-8, max_outer=5)
    o2.krylov_dim = 40
    with pytest.raises(ptp.PtpError):
        c2.newton_solve(o2)
