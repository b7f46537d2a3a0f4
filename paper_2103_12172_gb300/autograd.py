"""torch.autograd wrapper of the batched projection columns and their hand-written adjoint.

    out = project(plan, k, xi=None, kind="Q")

k: real tensor [n_subs] of per-subdomain wavenumbers (may require grad); xi: optional complex128
CUDA tensor of user densities (layout of the output, may require grad). The forward refactors
the plan when k differs from the plan's current wavenumbers (mdp_plan_update_k: every mode's
pivoted LU, dT/dk rows and sweep table rebuilt by the device factorisation kernels, only the
subdomain descriptors uploaded) and runs mdp_project_batch; the backward runs mdp_ap_adjoint
(conjugate-transposed AP solve, and the dG/dk second solve for the wavenumber gradient).
"""
from __future__ import annotations

import torch


def _set_k(plan, k):
    ks = [float(v) for v in k.detach().cpu().tolist()]
    if getattr(plan, "_k_current", None) != ks:
        plan.update_k(ks)
        plan._k_current = ks
    return ks


class MdpProject(torch.autograd.Function):
    @staticmethod
    def forward(ctx, k, xi, plan, kind):
        ks = _set_k(plan, k)
        out = plan.project(xi=xi, kind=kind)
        ctx.plan, ctx.kind, ctx.ks = plan, kind, ks
        ctx.save_for_backward(xi if xi is not None else torch.empty(0))
        ctx.has_xi = xi is not None
        ctx.k_meta = (k.dtype, k.device)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        plan = ctx.plan
        (xi,) = ctx.saved_tensors
        xi = xi if ctx.has_xi else None
        if getattr(plan, "_k_current", None) != ctx.ks:
            plan.update_k(ctx.ks)
            plan._k_current = ctx.ks
        want_xi = ctx.has_xi and ctx.needs_input_grad[1]
        want_k = ctx.needs_input_grad[0]
        gx, gk = plan.adjoint(grad_out.contiguous(), xi=xi, kind=ctx.kind, grad_xi=want_xi,
                              grad_k=torch.zeros(plan.n_subs, dtype=torch.float64, device=grad_out.device)
                              if want_k else None) if (want_xi or want_k) else (None, None)
        dtype, device = ctx.k_meta
        gk = gk.to(dtype=dtype, device=device) if (want_k and gk is not None) else None
        return gk, (gx if want_xi else None), None, None


def project(plan, k, xi=None, kind="Q"):
    return MdpProject.apply(k, xi, plan, kind)
