"""Differentiable rate-distortion loss of one image (Sec. IV-A, Eq. 10) for torch.autograd.

`rd_loss(latents, params, image, H=..., W=..., hp=...)` returns (loss, rate_bits, mse) as 0-dim
FP64 device tensors; `loss` carries gradients to `latents` and `params`.  The forward is
coolchic_forward and the backward is the library's hand-written adjoint, coolchic_backward:
there is no autograd tape inside, every step runs in the library's kernels.

recompute=True (default) keeps nothing between the two passes: the adjoint kernels recompute the
entropy-model and synthesis activations per tile.  recompute=False stores them in the workspace
during the forward (34 floats per latent, 40 per pixel) and the adjoint reads them back.
"""
from __future__ import annotations

import torch

from . import lib as cc


class _RDLoss(torch.autograd.Function):
    @staticmethod
    def forward(ctx, latents, params, image, H, W, hp, step, relax, recompute):
        dev = latents.device
        ws = cc.workspace(H, W, store_activations=not recompute, device=dev)
        rd = torch.empty(3, dtype=torch.float64, device=dev)
        cc.forward(image, latents.detach(), params.detach(), H=H, W=W, hp=hp, step=step, relax=relax, ws=ws,
                   store=not recompute, rd=rd)
        ctx.save_for_backward(latents, params, image)
        ctx.cfg = (H, W, hp, step, relax, recompute)
        ctx.ws = ws
        loss, rate, mse = rd[0], rd[1], rd[2]
        ctx.mark_non_differentiable(rate, mse)
        return loss, rate, mse

    @staticmethod
    def backward(ctx, g_loss, g_rate, g_mse):
        latents, params, image = ctx.saved_tensors
        H, W, hp, step, relax, recompute = ctx.cfg
        g_lat = torch.empty_like(latents)
        g_par = torch.empty_like(params)
        scale = 0.0 if g_loss is None else float(g_loss)  # dOut/dLoss enters the kernels as grad_scale
        cc.backward(image, latents.detach(), params.detach(), g_lat, g_par, H=H, W=W, hp=hp, step=step,
                    relax=relax, ws=ctx.ws, use_stored=not recompute, grad_scale=scale)
        ctx.ws = None
        return g_lat, g_par, None, None, None, None, None, None, None


def rd_loss(latents: torch.Tensor, params: torch.Tensor, image: torch.Tensor, *, H: int, W: int,
            hp: cc.HParams, step: int = 0, relax: int = cc.CC_RELAX_NOISE, recompute: bool = True):
    """(loss, rate_bits, mse) of the state (latents, params) on `image` (CHW FP32, device), with the
    latents relaxed as `relax` at `step` (the noise is keyed by hp.seed and step)."""
    for name, t in (("latents", latents), ("params", params), ("image", image)):
        if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
            raise ValueError(f"{name} must be a contiguous float32 CUDA tensor")
    return _RDLoss.apply(latents, params, image, H, W, hp, int(step), int(relax), bool(recompute))
