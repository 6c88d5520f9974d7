"""The smoothed potential of the MWU solver as a differentiable torch function.

pot(x) = smax_eta(P x) - smin_eta(C x), the potential of Sec. 4.1 without its
1/eta factor, evaluated on the device by the library (``mwu_potential``).  One
call returns the value and the three gradients:

* d pot / d x = P^T nabla smax(Px) - C^T nabla smin(Cx)      (= g - h of Alg. 2)
* d pot / d c for the objective row (1/M) c^T of a pure packing or covering LP
* d pot / d val for the stored values of an explicit CSR side
  (+w_j x_i on the packing side, -w_j x_i on the covering side)

The context fixes P, C, eta (``mwu_set_target``) and reads the objective and
the CSR values it was created from.  The tensors passed here for them must
hold the same values: ``potential`` checks them against the context's copies
on the device (``mwu_check_values``) and raises ValueError when they differ
(for instance after an in-place update), since the gradients refer to the
context's copies.  Every step runs in the library's kernels; there is no CPU
path.
"""
from __future__ import annotations

import torch

from . import mwu as M


class _Potential(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, objective, values, handle, n_values):
        if not x.is_cuda:
            raise ValueError("x must be a CUDA tensor")
        x32 = x.detach().to(torch.float32).contiguous()
        gx = torch.empty_like(x32)
        gobj = torch.empty_like(x32) if objective is not None else None
        gval = torch.empty(n_values, dtype=torch.float32, device=x.device) if values is not None else None
        pot = M.mwu_potential(handle, x32, gx, gobj, gval)
        ctx.grads = (gx, gobj, gval)
        ctx.dtypes = (x.dtype, None if objective is None else objective.dtype,
                      None if values is None else values.dtype)
        return torch.tensor(pot, dtype=torch.float64, device=x.device)

    @staticmethod
    def backward(ctx, gout):
        gx, gobj, gval = ctx.grads
        dx, dobj, dval = ctx.dtypes
        out_x = (gout * gx.double()).to(dx) if ctx.needs_input_grad[0] else None
        out_obj = (gout * gobj.double()).to(dobj) if (gobj is not None and ctx.needs_input_grad[1]) else None
        out_val = (gout * gval.double()).to(dval) if (gval is not None and ctx.needs_input_grad[2]) else None
        return out_x, out_obj, out_val, None, None


def potential(handle, x, objective=None, values=None):
    """pot(x) on the context ``handle`` (a target must be set); differentiable in x,
    ``objective`` (the c the context was created with) and ``values`` (the explicit
    CSR values it was created with, packing side first)."""
    n_values = int(values.numel()) if values is not None else 0
    if (objective is not None or values is not None) and not M.mwu_check_values(handle, objective, values):
        raise ValueError("objective / values differ from the arrays the context was created with; create a new "
                         "context for new values")
    return _Potential.apply(x, objective, values, handle, n_values)
