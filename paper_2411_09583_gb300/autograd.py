"""Differentiable NUHT: torch.autograd.Function over the C ABI.

    g = A(r, omega) c,   A(k, j) = J_nu(omega_k r_j)

backward, for an upstream gradient e = dL/dg:
    dL/dc     = A^T e                                      (nuht_adjoint)
    dL/dr_j   = c_j [A_{nu-1}^T (omega e) - A_{nu+1}^T (omega e)]_j / 2
    dL/domega = e [A_{nu-1} (r c) - A_{nu+1} (r c)] / 2
using J_nu' = (J_{nu-1} - J_{nu+1}) / 2 (DLMF 10.6.1) with plans of orders
nu - 1 and nu + 1 on the same points (J_{-1} = -J_1 is handled by the library).
Real c for the r / omega gradients; every transform runs in libnuht.so.
"""
import torch

from .nuht import Plan


class _NUHT(torch.autograd.Function):
    @staticmethod
    def forward(ctx, c, r, omega, nu, eps, opts):
        plan = Plan(nu, r.detach(), omega.detach(), eps, **opts)
        g = plan.execute(c.detach())
        ctx.save_for_backward(c, r, omega)
        ctx.plan, ctx.nu, ctx.eps, ctx.opts = plan, nu, eps, opts
        return g

    @staticmethod
    def backward(ctx, e):
        c, r, omega = ctx.saved_tensors
        e = e.contiguous()
        grad_c = grad_r = grad_w = None
        if ctx.needs_input_grad[0]:
            grad_c = ctx.plan.adjoint(e)
        if ctx.needs_input_grad[1] or ctx.needs_input_grad[2]:
            if c.is_complex():
                raise NotImplementedError("r / omega gradients are for real c")
            with Plan(ctx.nu - 1, r.detach(), omega.detach(), ctx.eps, **ctx.opts) as pm, \
                    Plan(ctx.nu + 1, r.detach(), omega.detach(), ctx.eps, **ctx.opts) as pp:
                if ctx.needs_input_grad[1]:
                    we = (omega.detach()[:, None] * e if e.dim() > 1 else omega.detach() * e).contiguous()
                    d = 0.5 * (pm.adjoint(we) - pp.adjoint(we))
                    grad_r = (c.detach() * d).reshape(c.shape[0], -1).sum(dim=1)
                if ctx.needs_input_grad[2]:
                    rc = (r.detach()[:, None] * c.detach() if c.dim() > 1 else r.detach() * c.detach())
                    d = 0.5 * (pm.execute(rc.contiguous()) - pp.execute(rc.contiguous()))
                    grad_w = (e * d).reshape(e.shape[0], -1).sum(dim=1)
        return grad_c, grad_r, grad_w, None, None, None


def nuht_autograd(c, r, omega, nu, eps, **opts):
    """g = A(r, omega) c with gradients for c, r and omega (all float64 CUDA tensors)."""
    return _NUHT.apply(c, r, omega, nu, eps, opts)
