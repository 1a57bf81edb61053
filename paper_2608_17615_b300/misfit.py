"""torch.autograd.Function for the far-field misfit of the differentiation form.

J(m) = 1/2 sum_r sum_a |u_inf^(r)(theta_a) - t_a^(r)|^2 over incident directions
r and receiver angles theta_a, with u^(r) solving L(m) u = b^(r)
(L = I + k^2 V diag(m)).  Forward: one preconditioned GMRES solve per
direction in the library; only u and the far-field residual are kept (the
Krylov bases are not, so nothing else is stored for the backward).  Backward:
the library's adjoint solve L^T lambda = m * A^T conj(res) and gradient
assembly (ls_misfit_gradient_dev).  m is the real nodal contrast.

batched=True runs the precision form for many directions: the forward solves
and the adjoint solves each advance all directions in lock step on the FP32
batched pair sum (ls_solve_batch_dev, ls_misfit_gradient_batch_dev).
"""
import numpy as np
import torch

from . import LS_ENOCONV


class FarFieldMisfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m, op, dir_angles, ff_angles, targets, batched=False):
        mh = m.detach().to("cpu", torch.float64).numpy().astype(np.complex128)
        op.set_contrast(mh)
        R = len(dir_angles)
        n = op.n
        b = torch.empty((R, n), dtype=torch.complex128, device=m.device)
        op.incident_dev(dir_angles, b)
        u = torch.empty_like(b)
        uinf = torch.empty((R, len(ff_angles)), dtype=torch.complex128, device=m.device)
        if batched:
            op.solve_batch_dev(b, u, ff_angles, uinf)
        else:
            op.solve_dev(b, u, ff_angles, uinf)
        resid = uinf - targets
        ctx.save_for_backward(u, resid)
        ctx.op, ctx.ff, ctx.batched = op, np.asarray(ff_angles, np.float64), batched
        r = resid.detach().cpu().numpy()
        return torch.tensor(0.5 * float(np.sum(np.abs(r) ** 2)), dtype=torch.float64, device=m.device)

    @staticmethod
    def backward(ctx, gJ):
        u, resid = ctx.saved_tensors
        grad = torch.empty(u.shape[-1], dtype=torch.float64, device=u.device)
        if ctx.batched:
            ctx.op.misfit_gradient_batch_dev(u, ctx.ff, resid.contiguous(), grad)
        else:
            ctx.op.misfit_gradient_dev(u, ctx.ff, resid.contiguous(), grad)
        return gJ * grad, None, None, None, None, None


def far_field_misfit(m, op, dir_angles, ff_angles, targets, batched=False):
    """J(m) as a differentiable scalar (see FarFieldMisfit)."""
    return FarFieldMisfit.apply(m, op, dir_angles, ff_angles, targets, batched)
