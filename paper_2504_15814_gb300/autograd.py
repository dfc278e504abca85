"""torch.autograd wrappers of the transfer operators.

Interpolate(coarse, fine, plan) returns a copy of ``fine`` whose fine ghost
halves hold P coarse; Restrict(fine, coarse, plan) returns a copy of
``coarse`` whose restricted halo volumes hold R fine (paper Sec. 2:
Q^f = P Q^c, Q^c = R Q^f).  Both maps are linear, so the backward passes
apply the transposed operators P^T and R^T (the library's adjoint kernels,
float64 in either precision mode); the gradient that flows through the
untouched entries is the upstream gradient with the written entries set to
zero.
"""
import torch


def _zeros(n, like):
    return torch.zeros(n, dtype=torch.float64, device=like.device)


class Interpolate(torch.autograd.Function):
    @staticmethod
    def forward(ctx, coarse, fine, plan):
        out = fine.detach().clone()
        plan.interpolate(coarse.detach().contiguous(), out)
        ctx.plan = plan
        return out

    @staticmethod
    def backward(ctx, g):
        plan = ctx.plan
        g = g.contiguous()
        g_coarse = g_fine = None
        if ctx.needs_input_grad[0]:
            g_coarse = torch.empty(plan.coarse_elems, dtype=torch.float64, device=g.device)
            plan.interpolate_adjoint(g, g_coarse)
        if ctx.needs_input_grad[1]:
            g_fine = g.clone()
            plan.interpolate(_zeros(plan.coarse_elems, g), g_fine)  # P 0 = 0 on the ghost entries
        return g_coarse, g_fine, None


class Restrict(torch.autograd.Function):
    @staticmethod
    def forward(ctx, fine, coarse, plan):
        out = coarse.detach().clone()
        plan.restrict(fine.detach().contiguous(), out)
        ctx.plan = plan
        return out

    @staticmethod
    def backward(ctx, g):
        plan = ctx.plan
        g = g.contiguous()
        g_fine = g_coarse = None
        if ctx.needs_input_grad[0]:
            g_fine = torch.empty(plan.fine_elems, dtype=torch.float64, device=g.device)
            plan.restrict_adjoint(g, g_fine)
        if ctx.needs_input_grad[1]:
            g_coarse = g.clone()
            plan.restrict(_zeros(plan.fine_elems, g), g_coarse)  # R 0 = 0 on the halo entries
        return g_fine, g_coarse, None


def interpolate(coarse, fine, plan):
    return Interpolate.apply(coarse, fine, plan)


def restrict(fine, coarse, plan):
    return Restrict.apply(fine, coarse, plan)
