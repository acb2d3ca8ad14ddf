"""torch.autograd.Function around the C ABI: the field H(m, t) and its gradients.

Forward: demag_apply.  Backward: demag_apply_adjoint for dLoss/dm (the
transposed-block convolution, A^T = D_t A D_t^-1) and demag_thickness_grad for
dLoss/dt_l of the layers whose thickness requires a gradient.  All arithmetic
runs in libdemag's kernels; this module only routes tensors.
"""
import torch

from . import _lib


class DemagField(torch.autograd.Function):
    """H = demag_field(m, thickness, plan, Ms, layers).

    m          CUDA tensor [B, L, 3, ny, nx] of the plan's dtype
    thickness  CPU float64 tensor [L], the plan's thicknesses (a leaf that may
               require grad; the plan must have been built from these values)
    plan       a paper_1910_07054_gb300.Plan
    Ms         saturation magnetization (A/m)
    layers     layer indices whose thickness gradient is computed (None: all)
    """

    @staticmethod
    def forward(ctx, m, thickness, plan, Ms, layers=None):
        H = plan.apply(m.contiguous(), Ms)
        ctx.plan = plan
        ctx.Ms = Ms
        ctx.layers = layers
        ctx.save_for_backward(m)
        return H

    @staticmethod
    def backward(ctx, gH):
        (m,) = ctx.saved_tensors
        plan, Ms = ctx.plan, ctx.Ms
        gH = gH.contiguous()
        gm = gt = None
        if ctx.needs_input_grad[0]:
            gm = torch.empty_like(gH)
            _lib.demag_apply_adjoint(plan.handle, gH, Ms, gm, info=plan.info)
        if ctx.needs_input_grad[1]:
            L = plan.info["L"]
            gt = torch.zeros(L, dtype=torch.float64)
            for layer in (range(L) if ctx.layers is None else ctx.layers):
                gt[layer] = _lib.demag_thickness_grad(plan.handle, m.contiguous(), gH, Ms, layer,
                                                      info=plan.info)
        return gm, gt, None, None, None


def demag_field(m, thickness, plan, Ms, layers=None):
    return DemagField.apply(m, thickness, plan, Ms, layers)
