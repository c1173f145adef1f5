"""torch.autograd.Function wrappers with hand-written backward passes.

The gradient of A is A^T, of A_S^dagger = (pi/m) B_S H is (pi/m) H B_S^T,
of T_g is T_g^T (Algorithm 2 differentiates ell_MC + lambda ell_SkEI with
respect to the network parameters; these are the operator-side factors of
that chain rule).  All forward and backward work runs in libskei's kernels;
torch only scales the incoming scalar gradient of the loss.
"""
from __future__ import annotations

import torch

from . import skei as S

__all__ = ["Proj", "FBP", "Rotate", "SkEIStage1", "SkEIFinish", "skei_loss"]


class Proj(torch.autograd.Function):
    """x [B, N, N] -> A_S x [B, m, n_det]."""

    @staticmethod
    def forward(ctx, x, plan, idx=None):
        ctx.plan, ctx.idx = plan, idx
        return S.proj_fwd(plan, x.contiguous(), idx)

    @staticmethod
    def backward(ctx, g):
        return S.proj_adj(ctx.plan, g.contiguous(), ctx.idx), None, None


class FBP(torch.autograd.Function):
    """p [B, m, n_det] -> A_S^dagger p [B, N, N]."""

    @staticmethod
    def forward(ctx, p, plan, idx=None):
        ctx.plan, ctx.idx = plan, idx
        return S.fbp(plan, p.contiguous(), idx)

    @staticmethod
    def backward(ctx, g):
        return S.fbp_adj(ctx.plan, g.contiguous(), ctx.idx), None, None


class Rotate(torch.autograd.Function):
    """x [B, N, N] -> T_g x [B, G, N, N] for g_deg [B, G] (float64, CUDA)."""

    @staticmethod
    def forward(ctx, x, g_deg):
        ctx.save_for_backward(g_deg)
        return S.rotate(x.contiguous(), g_deg)

    @staticmethod
    def backward(ctx, g):
        (g_deg,) = ctx.saved_tensors
        return S.rotate_adj(g.contiguous(), g_deg), None


class SkEIStage1(torch.autograd.Function):
    """x1 -> (r = S_mc y - A_mc x1, x2 = T_g x1, z = A_S^dagger A_S x2)."""

    @staticmethod
    def forward(ctx, x1, y, plan, g_deg, mc_idx=None, sk_idx=None):
        r, x2, z = S.ei_loss_fwd(plan, x1.contiguous(), y.contiguous(), g_deg, mc_idx, sk_idx)
        ctx.plan, ctx.mc_idx, ctx.sk_idx = plan, mc_idx, sk_idx
        ctx.save_for_backward(g_deg)
        return r, x2, z

    @staticmethod
    def backward(ctx, g_r, g_x2, g_z):
        (g_deg,) = ctx.saved_tensors
        plan = ctx.plan
        B, G = g_deg.shape
        like = (g_r if g_r is not None else g_x2 if g_x2 is not None else g_z)
        dev, dt = like.device, like.dtype
        mc_m = plan.n_angles if ctx.mc_idx is None else ctx.mc_idx.numel()
        if g_r is None:
            g_r = torch.zeros((B, mc_m, plan.n_det), device=dev, dtype=dt)
        if g_x2 is None:
            g_x2 = torch.zeros((B, G, plan.N, plan.N), device=dev, dtype=dt)
        if g_z is None:
            g_z = torch.zeros((B, G, plan.N, plan.N), device=dev, dtype=dt)
        # dr/dx1 = -A_mc: the library's MC term is -2 mc_coef A_mc^T (.), so
        # mc_coef = 1/2 applies -A_mc^T to the incoming g_r
        g_x1 = S.ei_loss_bwd(plan, g_r.contiguous(), g_x2.contiguous(), g_z.contiguous(), g_deg,
                             0.5, ctx.mc_idx, ctx.sk_idx)
        return g_x1, None, None, None, None, None


class SkEIFinish(torch.autograd.Function):
    """(x2, x3, r) -> loss = (1/B) sum_b [mc_scale ||r_b||^2 + lambda/G sum_g
    ||x2_bg - x3_bg||^2] (FP64 scalar)."""

    @staticmethod
    def forward(ctx, x2, x3, r, lam, mc_scale):
        loss, mc, ei, g_x2, g_x3 = S.ei_loss_finish(x2.contiguous(), x3.contiguous(),
                                                    r.contiguous(), lam, mc_scale)
        ctx.save_for_backward(g_x2, g_x3, r)
        ctx.rcoef = 2.0 * mc_scale / x2.shape[0]
        return loss.reshape(())

    @staticmethod
    def backward(ctx, gL):
        g_x2, g_x3, r = ctx.saved_tensors
        s = gL.to(g_x2.dtype)
        return g_x2 * s, g_x3 * s, r * (s * ctx.rcoef), None, None


def skei_loss(plan, x1, y, F, g_deg, mc_idx=None, sk_idx=None, lam=1.0, mc_scale=1.0):
    """Eq. (e:skeiloss) for measurements y and network output x1 = F(A^dagger y):
    MC on the angles mc_idx, EI with the sketch sk_idx (None = all angles)."""
    r, x2, z = SkEIStage1.apply(x1, y, plan, g_deg, mc_idx, sk_idx)
    x3 = F(z)
    return SkEIFinish.apply(x2, x3, r, lam, mc_scale)
