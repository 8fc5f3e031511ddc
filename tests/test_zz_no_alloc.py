"""ptp_residual_noalloc_dev: the outer residual for callers that cannot let
the library allocate device memory during the call (a framework whose own
pool owns the GPU, a hard memory budget, or a loop that cannot pay for the
synchronisation of cudaMalloc/cudaFree).  Its scratch is a fixed 4 MiB array
inside the library, so it must give the same R and ||R|| as the regular
ptp_residual_dev, call after call, leave the device's free memory unchanged,
and refuse problems whose iron fluxes do not fit.  This file is collected
last so that a run stopping at the first failure has already run every other
test."""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
ptp = pytest.importorskip("paper_2502_21013_gb300.ptp")

# iron element fluxes that fit the fixed scratch: 2 * n_iron * N <= LIMIT doubles
LIMIT = 522232


def _ctx(prob):
    c = ptp.Context(0)
    ptp.load_problem(c, prob)
    c.setup(ptp.default_opts(precision=ptp.PTP_FP64))
    return c


def _noalloc(c, U, R, nrm):
    p = lambda t: ctypes.c_void_p(t.data_ptr()) if t is not None else None
    rc = ptp.lib.ptp_residual_noalloc_dev(c._h, p(U), p(R), p(nrm))
    if rc != ptp.PTP_OK:
        raise ptp.PtpError(rc, ptp.lib.ptp_last_error(c._h).decode())


def _check_twice(prob, scales, seed):
    c = _ctx(prob)
    n, N = prob.n_free, prob.N
    rng = np.random.default_rng(seed)
    R_ref = torch.empty((n, N), dtype=torch.float64, device="cuda")
    R = torch.empty_like(R_ref)
    nrm = torch.zeros(1, dtype=torch.float64, device="cuda")
    for scale in scales:      # two calls in a row, different states
        U = torch.tensor(rng.normal(scale=scale, size=(n, N)), device="cuda")
        ref_norm = c.residual_dev(U, R_ref)
        R.fill_(float("nan"))
        nrm.fill_(float("nan"))
        _noalloc(c, U, R, nrm)
        torch.cuda.synchronize()
        err = (torch.linalg.norm(R - R_ref) / torch.linalg.norm(R_ref)).item()
        assert err < 1e-13
        assert abs(nrm.item() - ref_norm) <= 1e-13 * ref_norm
    return c


def test_noalloc_residual_matches_regular_entry_point_twice():
    _check_twice(W.config_plain_fp64(), (1e-2, 3.0), 11)   # 512 iron elements x 32 steps: fits


def test_noalloc_residual_with_the_exponential_law():
    """The iron fluxes of the law a min(exp(b s^2), c) + d (Section 4) go
    through the same scratch; states on both sides of the cap."""
    prob = W.paper_transformer_problem(21, 27, 6)
    assert 2 * int(np.count_nonzero(prob.nonlinear_e)) * prob.N <= LIMIT
    _check_twice(prob, (1e-6, 0.05), 3)


def test_noalloc_residual_optional_outputs_and_no_allocation():
    """R = NULL (norm only) and norm = NULL (R only) give the regular entry
    point's values, and after a first call the device's free memory does not
    change across calls."""
    prob = W.config_plain_fp64()
    c = _ctx(prob)
    n, N = prob.n_free, prob.N
    rng = np.random.default_rng(5)
    U = torch.tensor(rng.normal(scale=0.1, size=(n, N)), device="cuda")
    R_ref = torch.empty((n, N), dtype=torch.float64, device="cuda")
    ref_norm = c.residual_dev(U, R_ref)
    R = torch.empty_like(R_ref)
    nrm = torch.zeros(1, dtype=torch.float64, device="cuda")
    _noalloc(c, U, R, nrm)       # first call: symbol lookup, kernels loaded
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    nrm.fill_(float("nan"))
    _noalloc(c, U, None, nrm)    # norm only
    torch.cuda.synchronize()
    assert abs(nrm.item() - ref_norm) <= 1e-13 * ref_norm
    R.fill_(float("nan"))
    _noalloc(c, U, R, None)      # residual only
    torch.cuda.synchronize()
    assert (torch.linalg.norm(R - R_ref) / torch.linalg.norm(R_ref)).item() < 1e-13
    assert torch.cuda.mem_get_info()[0] == free0


def test_noalloc_residual_rejects_aliased_buffers():
    prob = W.config_plain_fp64()
    c = _ctx(prob)
    U = torch.zeros((prob.n_free, prob.N), dtype=torch.float64, device="cuda")
    R = torch.empty_like(U)
    for args in ((U, U, None), (U, R, U), (U, R, R)):
        with pytest.raises(ptp.PtpError) as e:
            _noalloc(c, *args)
        assert e.value.code == ptp.PTP_EINVAL


def test_noalloc_residual_size_limit_is_exact():
    """33x33 unit square: 512 iron elements; N = 509 needs 2 * 512 * 509 =
    521216 doubles (fits), N = 510 needs 522240 (one element-step too many)."""
    ok = W.unit_square_problem(33, 509)
    assert 2 * int(np.count_nonzero(ok.nonlinear_e)) * ok.N <= LIMIT
    _check_twice(ok, (0.5,), 7)
    big = W.unit_square_problem(33, 510)
    assert 2 * int(np.count_nonzero(big.nonlinear_e)) * big.N > LIMIT
    c = _ctx(big)
    U = torch.zeros((big.n_free, big.N), dtype=torch.float64, device="cuda")
    R = torch.empty_like(U)
    nrm = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(ptp.PtpError) as e:
        _noalloc(c, U, R, nrm)
    assert e.value.code == ptp.PTP_EINVAL and "scratch" in str(e.value)


def test_noalloc_residual_rejects_problems_beyond_the_scratch():
    prob = W.unit_square_problem(129, 64)   # 8192 iron elements x 64 steps > limit
    c = _ctx(prob)
    U = torch.zeros((prob.n_free, prob.N), dtype=torch.float64, device="cuda")
    R = torch.empty_like(U)
    nrm = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(ptp.PtpError) as e:
        _noalloc(c, U, R, nrm)
    assert e.value.code == ptp.PTP_EINVAL and "scratch" in str(e.value)
