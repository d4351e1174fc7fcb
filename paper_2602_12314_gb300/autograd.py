"""torch.autograd.Function wrappers around the hand-written forward/backward kernels.

SplatQueries:   f (N x d) -> Q (H*W x d)             Eq. (render_query); backward = latentam_render_bwd
DictDecodeLoss: (Q, K, V) -> lambda_f L_f (scalar)   Eq. (dict_recon) + Eq. (feat_loss); the forward
                computes the loss and its gradients in one pass (latentam_decode_loss_bwd), the
                backward scales them by the incoming gradient.
"""
from __future__ import annotations

import torch

from . import api


class SplatQueries(torch.autograd.Function):
    @staticmethod
    def forward(fctx, f, ctx: api.Context, proj: api.Projection, camera, bins: api.TileBins):
        Q, T, nc = api.render_fwd(ctx, proj, camera, bins, f.detach())
        fctx.lat = (ctx, proj, camera, bins)
        fctx.save_for_backward(nc)
        fctx.mark_non_differentiable(T, nc)
        return Q, T, nc

    @staticmethod
    def backward(fctx, dQ, _dT, _dnc):
        (nc,) = fctx.saved_tensors
        ctx, proj, camera, bins = fctx.lat
        df = api.render_bwd(ctx, proj, camera, bins, nc, dQ)
        return df, None, None, None, None


class DictDecodeLoss(torch.autograd.Function):
    @staticmethod
    def forward(fctx, Q, K, V, ctx: api.Context, V0, F, mask, cfg: api.LossConfig, precision: int):
        parts, dQ, dK, dV = api.decode_loss_bwd(ctx, Q.detach(), K.detach(), V.detach(), V0, F, mask, cfg, precision,
                                                need_dQ=Q.requires_grad)
        fctx.save_for_backward(*(t for t in (dQ, dK, dV) if t is not None))
        fctx.has_dQ = dQ is not None
        return parts[3].clone()

    @staticmethod
    def backward(fctx, g):
        saved = list(fctx.saved_tensors)
        dQ = saved.pop(0) if fctx.has_dQ else None
        dK, dV = saved
        s = g.to(torch.float32)
        return (dQ * s if dQ is not None else None), dK * s, dV * s, None, None, None, None, None, None


def latent_loss(f, K, V, ctx: api.Context, proj, camera, bins, V0, F, mask, cfg=None, precision=api.FP32):
    """lambda_f L_f of one keyframe as a differentiable function of (f, K, V)."""
    Q, _, _ = SplatQueries.apply(f, ctx, proj, camera, bins)
    return DictDecodeLoss.apply(Q, K, V, ctx, V0, F, mask, cfg or api.LossConfig(), precision)
