"""Arguments that would make the library read or write outside a caller's
buffer, or read a buffer it is writing, are rejected before any launch: a
block of the wrong size (binding) and aliased input and output (C ABI)."""
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
ptp = pytest.importorskip("paper_2502_21013_gb300.ptp")


def test_mis_sized_and_aliased_buffers_are_rejected():
    prob = W.unit_square_problem(9, 4)
    c = ptp.Context(0)
    ptp.load_problem(c, prob)
    c.setup(ptp.default_opts(precision=ptp.PTP_FP64))
    n, N = prob.n_free, prob.N
    X = torch.zeros((n, N), dtype=torch.float64, device="cuda")
    with pytest.raises(ptp.PtpError) as e:
        c.apply_shifted_dev(0, X, X)
    assert e.value.code == ptp.PTP_EINVAL
    with pytest.raises(ptp.PtpError) as e:
        c.apply_shifted_dev(0, X, torch.zeros((n, N - 1), dtype=torch.float64, device="cuda"))
    assert e.value.code == ptp.PTP_EINVAL
    for call in (lambda: c.residual_dev(X, X), lambda: c.spatial_solve_dev(0, X, X, 1e-6, 3),
                 lambda: c.periodic_solve_dev(X, X, 1), lambda: c.periodic_apply_dev(0, X, X),
                 lambda: c.solve_dev(torch.zeros(n * N + 1, dtype=torch.float64, device="cuda"))):
        with pytest.raises(ptp.PtpError) as e:
            call()
        assert e.value.code == ptp.PTP_EINVAL
    # the context is still usable: (M + tau L) 0 = 0
    Y = torch.full_like(X, 1.0)
    c.apply_shifted_dev(0, X, Y)
    torch.cuda.synchronize()
    assert int(torch.count_nonzero(Y)) == 0
    c.close()
