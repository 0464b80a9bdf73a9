"""Differentiable NUHT: torch.autograd.Function over the C ABI.

    g = A(r, omega) c,   A(k, j) = J_nu(omega_k r_j)

backward, for an upstream gradient e = dL/dg:
    dL/dc     = A^T e                                            (nuht_adjoint)
    dL/dr_j   = c_j sum_k e_k omega_k J_nu'(omega_k r_j)         (nuht_grad_r)
    dL/domega = e_k sum_j c_j r_j J_nu'(omega_k r_j)             (nuht_grad_omega)
with J_nu' = (J_{nu-1} - J_{nu+1}) / 2 (DLMF 10.6.1), through a derivative
plan of orders nu - 1 and nu + 1 built from the forward plan's sorted points
and frequencies (nuht_plan_deriv).  The weightings, the half difference and the
sum over vectors run in the library's kernels; this module only passes tensors.
Real c for the r / omega gradients.
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
            with ctx.plan.deriv() as d:
                if ctx.needs_input_grad[1]:
                    grad_r = d.grad_r(c.detach(), e)
                if ctx.needs_input_grad[2]:
                    grad_w = d.grad_omega(c.detach(), e)
        return grad_c, grad_r, grad_w, None, None, None


def nuht_autograd(c, r, omega, nu, eps, **opts):
    """g = A(r, omega) c with gradients for c, r and omega (all float64 CUDA tensors)."""
    return _NUHT.apply(c, r, omega, nu, eps, opts)
