"""torch.autograd.Function for the period-averaged eddy-current loss.

forward:  set the coil amplitudes, the iron law parameters and the element
          conductivities, solve Problem 1 (ptp_solve_dev) and evaluate the
          loss J (ptp_loss_dev).
backward: ptp_adjoint_gradient_dev at the converged state, scaled by the
          incoming gradient.
All arithmetic runs in libptp.so; this module only moves arguments.
"""
from __future__ import annotations

import torch

from . import ptp


class PeriodicLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, amp, nu_params, sigma, problem, opts=None, device=0):
        c = ptp.Context(device)
        prob = problem.replace(amp=amp.detach().cpu().double().numpy(),
                               nu_min=float(nu_params[0]), nu_max=float(nu_params[1]), s_sat=float(nu_params[2]),
                               sigma_e=sigma.detach().cpu().double().numpy())
        ptp.load_problem(c, prob)
        o = opts if opts is not None else ptp.default_opts(precision=ptp.PTP_FP64, tol=1e-12, max_outer=50000)
        c.setup(o)
        U = torch.zeros((prob.n_free, prob.N), dtype=torch.float64, device=f"cuda:{device}")
        st, rc = c.solve_dev(U, o)
        if rc != ptp.PTP_OK:
            # an unconverged state would give a loss and a gradient of the wrong problem
            raise ptp.PtpError(rc, f"forward solve did not converge ({st.outer_iterations} outer iterations, "
                                   f"relative residual {st.res_final / max(st.res0, 1e-300):.2e})")
        J = c.loss_dev(U)
        ctx.c, ctx.U, ctx.opts = c, U, o
        ctx.devices = (amp.device, nu_params.device, sigma.device)
        return torch.tensor(J, dtype=torch.float64)

    @staticmethod
    def backward(ctx, gJ):
        J, damp, dnu, dsig, st, rc = ctx.c.adjoint_gradient_dev(ctx.U, ctx.opts)
        if rc != ptp.PTP_OK:
            raise ptp.PtpError(rc, f"adjoint solve did not converge ({st.outer_iterations} outer iterations)")
        g = float(gJ)
        da = torch.tensor(damp, dtype=torch.float64, device=ctx.devices[0]) * g
        dn = torch.tensor(dnu, dtype=torch.float64, device=ctx.devices[1]) * g
        ds = dsig.to(ctx.devices[2]) * g
        return da, dn, ds, None, None, None


def periodic_loss(amp, nu_params, sigma, problem, opts=None, device=0):
    """J as a differentiable function of (amp, (nu_min, nu_max, s_sat), sigma)."""
    return PeriodicLoss.apply(amp, nu_params, sigma, problem, opts, device)
