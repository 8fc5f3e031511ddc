"""Adjoint gradient of the period-averaged eddy-current loss on the GPU,
against the oracle's adjoint (itself pinned by finite differences) and
against central differences of J(U(p)) computed on the GPU."""
import numpy as np
import pytest

import workloads as W
from oracle import adjoint as AD
from oracle import periodic as P

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
ptp = pytest.importorskip("paper_2502_21013_gb300.ptp")


def _problem(n=17, N=8):
    prob = W.config_adjoint(0, n=n, N=N)
    return prob.replace(amp=np.array([7000.0, 4500.0]), phase=np.array([0.0, 0.7]))


def _ctx(prob, **kw):
    c = ptp.Context(0)
    ptp.load_problem(c, prob)
    o = ptp.default_opts(**kw)
    c.setup(o)
    return c, o


def _solve(c, o, prob):
    U = torch.zeros((prob.n_free, prob.N), dtype=torch.float64, device="cuda")
    st, rc = c.solve_dev(U, o)
    assert rc == ptp.PTP_OK
    return U


def test_loss_matches_oracle():
    prob = _problem()
    d = P.assemble(prob)
    c, _ = _ctx(prob, precision=ptp.PTP_FP64)
    U = np.random.default_rng(0).normal(scale=0.05, size=(d.n, d.N))
    J = c.loss_dev(torch.tensor(U, device="cuda"))
    Jo = AD.objective(prob, d, U)
    assert abs(J - Jo) <= 1e-13 * abs(Jo)


@pytest.mark.parametrize("precision,bar", [("fp64", 1e-8), ("mixed", 1e-7)])
def test_adjoint_gradient_matches_oracle(precision, bar):
    prob = _problem()
    d = P.assemble(prob)
    Jo, damp_o, dnu_o, dsig_o, _ = AD.gradient(prob, d)
    prec = ptp.PTP_FP64 if precision == "fp64" else ptp.PTP_MIXED
    c, o = _ctx(prob, precision=prec, tol=1e-13 if precision == "fp64" else 1e-12, max_outer=50000)
    U = _solve(c, o, prob)
    J, damp, dnu, dsig, st, rc = c.adjoint_gradient_dev(U, o)
    assert rc == ptp.PTP_OK and st.converged
    assert abs(J - Jo) <= 1e-10 * abs(Jo)
    scale_nu = np.abs(dnu_o).max()
    assert np.abs(np.array(damp) - damp_o).max() <= bar * np.abs(damp_o).max()
    assert np.abs(np.array(dnu) - dnu_o).max() <= bar * scale_nu
    ds = dsig.cpu().numpy()
    assert np.abs(ds - dsig_o).max() <= bar * np.abs(dsig_o).max()


def test_adjoint_gradient_matches_gpu_central_differences():
    prob = _problem(n=17, N=16)
    opts = dict(precision=ptp.PTP_FP64, tol=1e-13, max_outer=50000)
    c, o = _ctx(prob, **opts)
    U = _solve(c, o, prob)
    J0, damp, dnu, dsig, st, rc = c.adjoint_gradient_dev(U, o)
    ds = dsig.cpu().numpy()

    def J_of(p):
        cc, oo = _ctx(p, **opts)
        return cc.loss_dev(_solve(cc, oo, p))

    iron = np.flatnonzero(prob.nonlinear_e)
    e = int(iron[len(iron) // 2])
    cases = [
        (lambda p, v: p.replace(amp=np.array([v, p.amp[1]])), prob.amp[0], damp[0]),
        (lambda p, v: p.replace(nu_max=v), prob.nu_max, dnu[1]),
        (lambda p, v: p.replace(s_sat=v), prob.s_sat, dnu[2]),
        (lambda p, v: p.replace(sigma_e=np.where(np.arange(p.n_tri) == e, v, p.sigma_e)), prob.sigma_e[e], ds[e]),
    ]
    for setter, p0, grad in cases:
        h = 1e-6 * max(1.0, abs(p0))
        fd = (J_of(setter(prob, p0 + h)) - J_of(setter(prob, p0 - h))) / (2 * h)
        assert abs(fd - grad) <= 1e-5 * max(abs(fd), 1e-6 * abs(J0)), (p0, fd, grad)


def test_autograd_function_backward_is_the_adjoint():
    from paper_2502_21013_gb300.autograd import periodic_loss
    prob = _problem(n=9, N=8)
    amp = torch.tensor(prob.amp, dtype=torch.float64, requires_grad=True)
    nu = torch.tensor([prob.nu_min, prob.nu_max, prob.s_sat], dtype=torch.float64, requires_grad=True)
    sig = torch.tensor(prob.sigma_e, dtype=torch.float64, requires_grad=True)
    J = periodic_loss(amp, nu, sig, prob)
    J.backward()
    Jo, damp_o, dnu_o, dsig_o, _ = AD.gradient(prob)
    assert abs(J.item() - Jo) <= 1e-9 * abs(Jo)
    assert np.abs(amp.grad.numpy() - damp_o).max() <= 1e-7 * np.abs(damp_o).max()
    assert np.abs(nu.grad.numpy() - dnu_o).max() <= 1e-7 * np.abs(dnu_o).max()
    assert np.abs(sig.grad.numpy() - dsig_o).max() <= 1e-7 * np.abs(dsig_o).max()


def test_autograd_function_raises_on_an_unconverged_solve():
    """A forward solve stopped by max_outer is not the solution of the problem,
    so neither its loss nor a gradient at it may be returned."""
    from paper_2502_21013_gb300.autograd import periodic_loss
    prob = _problem(n=9, N=8)
    amp = torch.tensor(prob.amp, dtype=torch.float64, requires_grad=True)
    nu = torch.tensor([prob.nu_min, prob.nu_max, prob.s_sat], dtype=torch.float64, requires_grad=True)
    sig = torch.tensor(prob.sigma_e, dtype=torch.float64, requires_grad=True)
    opts = ptp.default_opts(precision=ptp.PTP_FP64, tol=1e-12, max_outer=2)
    with pytest.raises(ptp.PtpError) as e:
        periodic_loss(amp, nu, sig, prob, opts)
    assert e.value.code == ptp.PTP_ENOTCONV
