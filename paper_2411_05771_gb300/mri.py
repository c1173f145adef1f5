"""Coil-sketched EI for multi-coil MRI (Sec. 3.4, Algorithm 3) on libskei.

Set-up, once per measurement y (k-space of N_c coils): PCA coil compression
to L virtual coils, then the coil sketch S_c = [I_R 0; 0 S_low] with a
Rademacher S_low, folded into one complex mixing W = S_c Q_L^T [M_c, N_c]
that forms both the sketched data y_S = W y and the sketched maps
C_S = W C (virtual coil l is sum_c Q[c, l] k_c = M F((sum_c Q[c, l] C_c) x), so
the compressed maps follow from the known maps; the paper estimates them
with ESPIRiT).  The covariance is one GEMM (cuBLAS) and the eigenvectors
come from cuSOLVER, both in FP64; the mixing, the operators and every step
of the iteration run in libskei's kernels.

A step (``CskArm.step``) is Algorithm 3's iteration with the residual
stand-in network F(u) = u + theta, and the transforms T_g rotations of both
planes of the complex image.
"""
from __future__ import annotations

import numpy as np
import torch

from . import skei as S

__all__ = ["coil_pca", "coil_sketch_mixing", "CoilSketch", "CskArm"]


def coil_pca(k: torch.Tensor, L: int) -> torch.Tensor:
    """Q_L [N_c, L] (complex128) of one measurement's k-space k [N_c, 2, N, N]:
    the L dominant eigenvectors of the coils' centred covariance
    V_ij = conj(kbar_i) . kbar_j / (d - 1), each with its largest-magnitude
    entry (the first such) made real positive."""
    Nc = k.shape[0]
    K = torch.complex(k[:, 0].double(), k[:, 1].double()).reshape(Nc, -1)   # [Nc, d]
    Kb = K - K.mean(dim=1, keepdim=True)
    V = (Kb.conj() @ Kb.T) / (K.shape[1] - 1)
    w, Q = torch.linalg.eigh(V)
    order = torch.argsort(-w, stable=True)
    Q = Q[:, order][:, :L]
    i = torch.argmax(Q.abs(), dim=0)
    piv = Q[i, torch.arange(L, device=Q.device)]
    return Q * (piv.conj() / piv.abs())[None, :]


def coil_sketch_mixing(Q: torch.Tensor, R: int, s_low: np.ndarray) -> torch.Tensor:
    """W = S_c Q_L^T [M_c, N_c] with S_c = [[I_R, 0], [0, S_low]]."""
    L = Q.shape[1]
    s_low = np.asarray(s_low, dtype=np.float64)
    Mc = R + s_low.shape[0]
    Sc = np.zeros((Mc, L))
    Sc[:R, :R] = np.eye(R)
    Sc[R:, R:] = s_low
    return torch.tensor(Sc, dtype=torch.complex128, device=Q.device) @ Q.T


class CoilSketch:
    """Sketched maps C_S, data y_S and dinv_S of one measurement."""

    def __init__(self, y: torch.Tensor, maps: torch.Tensor, L: int, R: int, s_low):
        self.Q = coil_pca(y[0], L)
        self.W = coil_sketch_mixing(self.Q, R, s_low).to(torch.complex64)
        self.maps = S.coil_mix(self.W, maps[None])[0].contiguous()
        self.y = S.coil_mix(self.W, y)
        self.dinv = S.mri_dinv(self.maps)


class CskArm:
    """One measurement's EI iteration on resident buffers: `maps`, `y`,
    `dinv` are the operator the loss uses (the full coils for EI, the coil
    sketch for C-SkEI, a coil subset for SkEI); x0 = A^dagger y of the full
    acquisition."""

    launches_per_step = 22

    def __init__(self, x0, y, maps, mask, dinv, G: int, lam: float = 1.0, lr: float = 5e-4):
        dev = x0.device
        N = x0.shape[-1]
        Mc = maps.shape[0]
        self.x0, self.y, self.maps, self.mask, self.dinv = x0, y, maps, mask, dinv
        self.G, self.lam, self.lr, self.N, self.Mc = G, lam, lr, N, Mc
        f32 = dict(dtype=torch.float32, device=dev)
        self.theta = torch.zeros((2, N, N), **f32)
        self.m1 = torch.zeros_like(self.theta)
        self.v1 = torch.zeros_like(self.theta)
        self.g = torch.zeros((1, G), dtype=torch.float64, device=dev)
        self.step_no = torch.ones((), dtype=torch.int32, device=dev)
        self.x1 = torch.empty((1, 2, N, N), **f32)
        self.r = torch.empty((1, Mc, 2, N, N), **f32)
        self.x2 = torch.empty((1, G, 2, N, N), **f32)
        self.p = torch.empty((G, Mc, 2, N, N), **f32)
        self.z = torch.empty((G, 2, N, N), **f32)
        self.x3 = torch.empty((1, G, 2, N, N), **f32)
        self.gx1 = torch.empty((1, 2, N, N), **f32)
        self.gx2 = torch.empty_like(self.x2)
        self.gx3 = torch.empty_like(self.x2)
        self.loss = torch.empty(1, dtype=torch.float64, device=dev)
        self.mc = torch.empty(1, dtype=torch.float64, device=dev)
        self.ei = torch.empty((1, G), dtype=torch.float64, device=dev)
        nb = max(S.mri_workspace_size(N, Mc, G), S.mri_workspace_size(N, Mc, 1), 16)
        self.work = torch.empty(nb, dtype=torch.uint8, device=dev)

    def grad(self):
        """Loss and dL/dx1 (in gx1), dL/dx3 (in gx3) for the current theta and g."""
        m, d, W, G, N = self.maps, self.mask, self.work, self.G, self.N
        S.residual_add(self.x0, self.theta, out=self.x1)                       # x1 = F(x0)
        S.mri_fwd(self.x1, m, d, aux=self.y, out=self.r, work=W)               # r = y - A x1
        S.rotate(self.x1, self.g, out=self.x2)                                 # x2 = T_g x1
        S.mri_fwd(self.x2.view(G, 2, N, N), m, d, out=self.p, work=W)
        S.mri_adj(self.p, m, d, self.dinv, out=self.z, work=W)                 # z = A^+ A x2
        S.residual_add(self.z, self.theta, out=self.x3.view(G, 2, N, N))       # x3 = F(z)
        S.ei_loss_finish(self.x2, self.x3, self.r, self.lam, 1.0, work=W,
                         out=(self.loss, self.mc, self.ei, self.gx2, self.gx3))
        # g_x2 += (A^+ A)^H g_z = A^H A (dinv g_z), g_z = g_x3 (F's Jacobian is I)
        S.mri_fwd(self.gx3.view(G, 2, N, N), m, d, xw=self.dinv, out=self.p, work=W)
        S.mri_adj(self.p, m, d, beta=1.0, out=self.gx2.view(G, 2, N, N), work=W)
        S.mri_adj(self.r, m, d, alpha=-2.0, out=self.gx1, work=W)               # -2 A^H r
        S.rotate_adj(self.gx2, self.g, beta=1.0, out=self.gx1)                 # + sum_g T_g^T

    def step(self):
        self.grad()
        # dL/dtheta = dL/dx1 + sum_g dL/dx3
        S.adam_step(self.theta, self.m1, self.v1, self.step_no, self.gx1, self.gx3, lr=self.lr)
