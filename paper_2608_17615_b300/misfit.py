"""torch.autograd.Function for the far-field misfit of the differentiation form.

J(m) = 1/2 sum_r sum_a |u_inf^(r)(theta_a) - t_a^(r)|^2 over incident directions
r and receiver angles theta_a, with u^(r) solving L(m) u = b^(r)
(L = I + k^2 V diag(m)).  Forward: one preconditioned GMRES solve per
direction in the library; only u and the far-field residual are kept (the
Krylov bases are not, so nothing else is stored for the backward).  Backward:
the library's adjoint solve L^T lambda = m * A^T conj(res) and gradient
assembly (ls_misfit_gradient_dev).  m is the real nodal contrast.
"""
import numpy as np
import torch

from . import LS_ENOCONV


class FarFieldMisfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m, op, dir_angles, ff_angles, targets):
        mh = m.detach().to("cpu", torch.float64).numpy().astype(np.complex128)
        op.set_contrast(mh)
        R = len(dir_angles)
        n = op.n
        b = torch.empty((R, n), dtype=torch.complex128, device=m.device)
        op.incident_dev(dir_angles, b)
        u = torch.empty_like(b)
        uinf = torch.empty((R, len(ff_angles)), dtype=torch.complex128, device=m.device)
        op.solve_dev(b, u, ff_angles, uinf)
        resid = uinf - targets
        ctx.save_for_backward(u, resid)
        ctx.op, ctx.ff = op, np.asarray(ff_angles, np.float64)
        r = resid.detach().cpu().numpy()
        return torch.tensor(0.5 * float(np.sum(np.abs(r) ** 2)), dtype=torch.float64, device=m.device)

    @staticmethod
    def backward(ctx, gJ):
        u, resid = ctx.saved_tensors
        grad = torch.empty(u.shape[-1], dtype=torch.float64, device=u.device)
        ctx.op.misfit_gradient_dev(u, ctx.ff, resid.contiguous(), grad)
        return gJ * grad, None, None, None, None


def far_field_misfit(m, op, dir_angles, ff_angles, targets):
    """J(m) as a differentiable scalar (see FarFieldMisfit)."""
    return FarFieldMisfit.apply(m, op, dir_angles, ff_angles, targets)
