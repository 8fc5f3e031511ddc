"""ptp_residual_noalloc_dev: the outer residual for callers that cannot let
the library allocate device memory during the call (a framework whose own
pool owns the GPU, a hard memory budget, or a loop that cannot pay for the
synchronisation of cudaMalloc/cudaFree).  Its scratch is a fixed 4 MiB array
inside the library, so it must give the same R and ||R|| as the regular
ptp_residual_dev, call after call, and refuse problems whose iron fluxes do
not fit.  This file is collected last so that a run stopping at the first
failure has already run every other test."""
import ctypes

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
ptp = pytest.importorskip("paper_2502_21013_gb300.ptp")


def _ctx(prob):
    c = ptp.Context(0)
    ptp.load_problem(c, prob)
    c.setup(ptp.default_opts(precision=ptp.PTP_FP64))
    return c


def _noalloc(c, U, R, nrm):
    p = lambda t: ctypes.c_void_p(t.data_ptr())
    rc = ptp.lib.ptp_residual_noalloc_dev(c._h, p(U), p(R), p(nrm))
    if rc != ptp.PTP_OK:
        raise ptp.PtpError(rc, ptp.lib.ptp_last_error(c._h).decode())


def test_noalloc_residual_matches_regular_entry_point_twice():
    prob = W.config_plain_fp64()   # 512 iron elements x 32 steps: fits the scratch
    c = _ctx(prob)
    n, N = prob.n_free, prob.N
    rng = np.random.default_rng(11)
    R_ref = torch.empty((n, N), dtype=torch.float64, device="cuda")
    R = torch.empty_like(R_ref)
    nrm = torch.zeros(1, dtype=torch.float64, device="cuda")
    for scale in (1e-2, 3.0):      # two calls in a row, different states
        U = torch.tensor(rng.normal(scale=scale, size=(n, N)), device="cuda")
        ref_norm = c.residual_dev(U, R_ref)
        R.fill_(float("nan"))
        _noalloc(c, U, R, nrm)
        torch.cuda.synchronize()
        err = (torch.linalg.norm(R - R_ref) / torch.linalg.norm(R_ref)).item()
        assert err < 1e-13
        assert abs(nrm.item() - ref_norm) <= 1e-13 * ref_norm


def test_noalloc_residual_rejects_problems_beyond_the_scratch():
    prob = W.unit_square_problem(129, 64)   # 8192 iron elements x 64 steps > limit
    c = _ctx(prob)
    U = torch.zeros((prob.n_free, prob.N), dtype=torch.float64, device="cuda")
    R = torch.empty_like(U)
    nrm = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(ptp.PtpError) as e:
        _noalloc(c, U, R, nrm)
    assert e.value.code == ptp.PTP_EINVAL and "scratch" in str(e.value)
