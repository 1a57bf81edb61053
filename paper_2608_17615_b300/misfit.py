"""torch.autograd.Function for the far-field misfit of the differentiation form.

J(m) = 1/2 sum_r sum_a |u_inf^(r)(theta_a) - t_a^(r)|^2 over incident directions
r and receiver angles theta_a, with u^(r) solving L(m) u = b^(r)
(L = I + k^2 V diag(m)).  Forward: the contrast goes to the library from the
device (ls_op_set_contrast_dev), one preconditioned GMRES solve per direction,
the misfit J and the far-field residual by the library (ls_misfit_dev); only u
and the residual are kept (the Krylov bases are not, so nothing else is stored
for the backward).  Backward: the library's adjoint solve
L^T lambda = m * A^T conj(res) and gradient assembly (ls_misfit_gradient_dev).
m is the real nodal contrast.  A solve that ends with LS_ENOCONV raises a
RuntimeWarning: the value and gradient then belong to an unconverged iterate.

batched=True runs the precision form for many directions: the forward solves
and the adjoint solves each advance all directions in lock step on the FP32
batched pair sum (ls_solve_batch_dev, ls_misfit_gradient_batch_dev).
"""
import warnings

import numpy as np
import torch

from . import LS_ENOCONV


def _warn_if_unconverged(st, what):
    if st == LS_ENOCONV:
        warnings.warn(f"{what}: GMRES reached max_iter or its explicit residual check failed; "
                      "the misfit and gradient come from an unconverged iterate", RuntimeWarning, stacklevel=3)


class FarFieldMisfit(torch.autograd.Function):
    @staticmethod
    def forward(ctx, m, op, dir_angles, ff_angles, targets, batched=False):
        op.set_contrast_dev(m.detach().contiguous())
        R = len(dir_angles)
        n = op.n
        b = torch.empty((R, n), dtype=torch.complex128, device=m.device)
        op.incident_dev(dir_angles, b)
        u = torch.empty_like(b)
        uinf = torch.empty((R, len(ff_angles)), dtype=torch.complex128, device=m.device)
        if batched:
            _, st = op.solve_batch_dev(b, u, ff_angles, uinf)
        else:
            _, st = op.solve_dev(b, u, ff_angles, uinf)
        _warn_if_unconverged(st, "forward solve")
        resid = torch.empty_like(uinf)
        J = op.misfit_dev(uinf, targets.contiguous(), resid)
        ctx.save_for_backward(u, resid)
        ctx.op, ctx.ff, ctx.batched = op, np.asarray(ff_angles, np.float64), batched
        return torch.tensor(J, dtype=torch.float64, device=m.device)

    @staticmethod
    def backward(ctx, gJ):
        u, resid = ctx.saved_tensors
        grad = torch.empty(u.shape[-1], dtype=torch.float64, device=u.device)
        if ctx.batched:
            _, st = ctx.op.misfit_gradient_batch_dev(u, ctx.ff, resid.contiguous(), grad)
        else:
            _, st = ctx.op.misfit_gradient_dev(u, ctx.ff, resid.contiguous(), grad)
        _warn_if_unconverged(st, "adjoint solve")
        return gJ * grad, None, None, None, None, None


def far_field_misfit(m, op, dir_angles, ff_angles, targets, batched=False):
    """J(m) as a differentiable scalar (see FarFieldMisfit)."""
    return FarFieldMisfit.apply(m, op, dir_angles, ff_angles, targets, batched)
