"""torch.autograd wrapper of the projection and its hand-written adjoint.

Forward: ``pressure_correct`` (Method III, Algorithm 1 of arXiv:2005.11806).
Backward: ``pressure_solve_adjoint`` (the transposed fixed-point system solved
by the same loop).  Marshalling only: both directions run in the CUDA
library; this module allocates the output tensors and passes pointers.
"""
from __future__ import annotations

import torch

from . import pressure as pp


class ProjectFunction(torch.autograd.Function):
    """(u*, v*, w*, rho) -> (u, v, w, p) with gradients w.r.t. u*, v*, w*, rho.

    ``plan`` is a ``pressure.Plan``; ``S`` (divergence target) is not
    differentiated.  Wall planes of w are not unknowns: their gradient is 0.
    """

    @staticmethod
    def forward(ctx, us, vs, ws, rho, plan, S, dt, rtol, maxit):
        p = torch.empty_like(rho)
        u, v = torch.empty_like(us), torch.empty_like(vs)
        w = torch.empty_like(ws)
        info = pp.pressure_correct(plan.handle, us, vs, ws, rho, S, dt, p, u, v, w,
                                   rtol=rtol, maxit=maxit)
        ctx.save_for_backward(rho, p)
        ctx.plan, ctx.dt, ctx.rtol, ctx.maxit = plan, dt, rtol, maxit
        ctx.info = info
        ctx.mark_non_differentiable(p)
        return u, v, w, p

    @staticmethod
    def backward(ctx, gu, gv, gw, gp):
        rho, p = ctx.saved_tensors
        gu = torch.zeros_like(p) if gu is None else gu.contiguous()
        gv = torch.zeros_like(p) if gv is None else gv.contiguous()
        if gw is None:
            gw = torch.zeros((p.shape[0] + 1,) + tuple(p.shape[1:]), dtype=p.dtype, device=p.device)
        else:
            gw = gw.contiguous()
        gus, gvs = torch.empty_like(gu), torch.empty_like(gv)
        gws, grho = torch.empty_like(gw), torch.empty_like(rho)
        pp.pressure_solve_adjoint(ctx.plan.handle, rho, p, ctx.dt, gu, gv, gw, gus, gvs, gws, grho,
                                  rtol=ctx.rtol, maxit=ctx.maxit)
        return gus, gvs, gws, grho, None, None, None, None, None


def project(us, vs, ws, rho, plan, S=None, dt=1e-3, rtol=1e-12, maxit=5000):
    """Differentiable projection: returns (u, v, w, p)."""
    return ProjectFunction.apply(us, vs, ws, rho, plan, S, dt, rtol, maxit)
