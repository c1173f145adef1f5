"""BN-only test-time training (Sec. 3.3): a residual CNN whose batch-norm
layers run in libskei's kernels, and whose only adapted parameters are the
BN layers' affine (scale, shift) pairs.

The paper adapts a pre-trained residual U-Net; neither it nor its weights
are available, so ``ResCNN`` stands in: 3x3 convolutions (frozen, seeded
weights from ``inputs.cnn_weights``; torch's cuDNN convolutions, the one
library step), each but the last followed by a batch-statistics BN layer
with ReLU (``skei_bn_act_fwd`` / ``skei_bn_act_bwd``), and a residual
connection F(u) = u + h(u).  The BN statistics are those of the batch the
network is applied to: the B measurements for x1 = F(A^dagger y), the B G
transformed reconstructions for x3 = F(z).
"""
from __future__ import annotations

import torch
import torch.nn.functional as tf

from . import skei as S
from .inputs import CnnWeights

__all__ = ["BNAct", "ResCNN"]


class BNAct(torch.autograd.Function):
    """v [B, C, ...] -> act(scale (v - mean) rstd + shift) with batch statistics."""

    @staticmethod
    def forward(ctx, v, scale, shift, relu=True, eps=1e-5):
        v = v.contiguous()
        out, mean, rstd = S.bn_act_fwd(v, scale, shift, relu, eps)
        ctx.save_for_backward(v, scale, shift, mean, rstd)
        ctx.relu = relu
        return out

    @staticmethod
    def backward(ctx, g):
        v, scale, shift, mean, rstd = ctx.saved_tensors
        g_v, g_scale, g_shift = S.bn_act_bwd(v, g.contiguous(), scale, shift, mean, rstd,
                                             ctx.relu)
        return g_v, g_scale, g_shift, None, None


class ResCNN:
    """F(u) = u + h(u) on images u [..., N, N] (every image one batch entry
    of one channel); ``bn`` (float32, requires grad) holds per BN layer its
    scale[C] then shift[C] and is the only parameter BN-only TTT adapts."""

    def __init__(self, weights: CnnWeights, device="cuda", eps: float = 1e-5):
        self.conv = [torch.tensor(w, dtype=torch.float32, device=device) for w in weights.conv]
        self.bn = torch.tensor(weights.bn, dtype=torch.float32, device=device).requires_grad_()
        self.C, self.L, self.eps = weights.channels, weights.layers, eps

    def parameters(self):
        return [self.bn]

    def __call__(self, u: torch.Tensor) -> torch.Tensor:
        N = u.shape[-1]
        h = u.reshape(-1, 1, u.shape[-2], N)
        C = self.C
        for l, w in enumerate(self.conv):
            h = tf.conv2d(h, w, padding=1)
            if l < self.L - 1:
                o = 2 * C * l
                h = BNAct.apply(h, self.bn[o:o + C], self.bn[o + C:o + 2 * C], True, self.eps)
        return u + h.reshape(u.shape)
