"""Numerical probe of Theorem 1 (the approximation bound of the sketched EI
regulariser) on a small explicit operator.

With F = identity (Lipschitz constant L = 1) and v of norm r, Theorem 1
sandwiches the mean over the N_S interleaved sketches S_k of
||v - A_S^+ A_S v|| between ||v - A^+ A v|| -+ r delta.  The proof bounds the
gap by ||A^+ (S^T S - I) A v||, then by (s_1 / s_k) ||U^T (S^T S - I) U|| r
with A = U Sigma V^T (rank k).  Here S_k selects the angles
{k, k + N_S, ...} of an n-angle sinogram, scaled so that the mean of S^T S
over the N_S offsets is I (S^T S = N_S P_k, P_k the selected rows).

The probe builds A column by column with libskei's Joseph projector (the
N^2 basis images in one batched launch), then uses torch.linalg (cuSOLVER,
FP64) for the SVD and the spectral norms, and libskei's FBP for the
regulariser as the experiments compute it (A^dagger = FBP, Sec. 2.1).
"""
from __future__ import annotations

import numpy as np
import torch

from . import skei as S
from .inputs import sketch_indices

__all__ = ["explicit_matrix", "theorem1"]


def explicit_matrix(plan: S.Plan, idx=None, batch: int = 1024) -> torch.Tensor:
    """A (or A_S for the int32 CUDA sketch idx) as a dense [m n_det, N^2]
    FP32 matrix: column j = A e_j, from the library's forward projector."""
    N = plan.N
    d = N * N
    m = plan.n_angles if idx is None else idx.numel()
    cols = []
    for j0 in range(0, d, batch):
        nb = min(batch, d - j0)
        e = torch.zeros((nb, d), dtype=torch.float32, device="cuda")
        e[torch.arange(nb, device="cuda"), torch.arange(j0, j0 + nb, device="cuda")] = 1.0
        p = S.proj_fwd(plan, e.view(nb, N, N), idx)
        cols.append(p.reshape(nb, m * plan.n_det))
    return torch.cat(cols).T.contiguous()


def _row_mask(n_angles: int, n_det: int, angles, device):
    mask = torch.zeros(n_angles, dtype=torch.float64, device=device)
    mask[torch.as_tensor(angles, device=device, dtype=torch.long)] = 1.0
    return mask.repeat_interleave(n_det)


def theorem1(plan: S.Plan, ns_list=(2, 5, 10, 20), v=None, rank_tol: float = 1e-10):
    """delta = max_k ||U^T (N_S P_k - I) U||_2 for each N_S in ns_list, with
    the numerical checks of the bound on the test images v [n, N, N] (F =
    identity): the proof's inequality, the theorem's sandwich with exact
    pseudo-inverses, and the FBP form of the regulariser."""
    N, n, nd = plan.N, plan.n_angles, plan.n_det
    A = explicit_matrix(plan).double()
    U, sig, Vh = torch.linalg.svd(A, full_matrices=False)
    k = int((sig > rank_tol * sig[0]).sum())
    U, sig, Vh = U[:, :k], sig[:k], Vh[:k]
    kappa = float(sig[0] / sig[-1])
    Apinv = Vh.T @ torch.diag(1.0 / sig) @ U.T                    # A^+
    out = {"N": N, "n_angles": n, "n_det": nd, "rank": k, "sigma_1": float(sig[0]),
           "sigma_k": float(sig[-1]), "kappa": kappa, "sketches": []}
    vv = None if v is None else v.reshape(v.shape[0], -1).double().T  # [d, n_v]
    if vv is not None:
        r = vv.norm(dim=0)
        e_ei = (vv - Apinv @ (A @ vv)).norm(dim=0)                  # ||v - A^+ A v||
        v32 = v.float().contiguous()
        fbp_full = S.fbp(plan, S.proj_fwd(plan, v32)).reshape(v.shape[0], -1).double().T
        e_fbp = (vv - fbp_full).norm(dim=0)
    for ns in ns_list:
        if n % ns:
            raise ValueError(f"N_S = {ns} does not divide {n} angles")
        m = n // ns
        deltas, chain, s_pinv, s_fbp = [], [], [], []
        for o in range(ns):
            ang = sketch_indices(n, m, o)
            mask = _row_mask(n, nd, ang, A.device)
            M = ns * (U.T * mask) @ U - torch.eye(k, dtype=torch.float64, device=A.device)
            dk = float(torch.linalg.eigvalsh(M).abs().max())
            deltas.append(dk)
            if vv is None:
                continue
            # the proof's chain: ||A^+ (N_S P - I) A v|| <= kappa delta_k ||v||
            w = Apinv @ ((ns * mask - 1.0)[:, None] * (A @ vv))
            chain.append(float((w.norm(dim=0) / (kappa * dk * r)).max()))
            # the theorem's A_S^+ A_S: the exact pseudo-inverse of the sketch
            rows = mask > 0
            As = A[rows]
            s_pinv.append((vv - torch.linalg.pinv(As, rtol=rank_tol) @ (As @ vv)).norm(dim=0))
            idx = torch.as_tensor(ang, dtype=torch.int32, device="cuda")
            zs = S.fbp(plan, S.proj_fwd(plan, v32, idx), idx).reshape(v.shape[0], -1)
            s_fbp.append((vv - zs.double().T).norm(dim=0))
        item = {"N_S": ns, "m": m, "delta_max": max(deltas),
                "delta_mean": float(np.mean(deltas))}
        if vv is not None:
            mean_pinv = torch.stack(s_pinv).mean(dim=0)
            mean_fbp = torch.stack(s_fbp).mean(dim=0)
            bound = kappa * item["delta_max"] * r
            item.update({
                "proof_chain_max_ratio": max(chain),
                "sandwich_holds": bool(((mean_pinv - e_ei).abs() <= bound).all()),
                "sandwich_gap_over_bound_max": float(((mean_pinv - e_ei).abs() / bound).max()),
                "ei_pinv_mean": float(e_ei.mean()), "skei_pinv_mean": float(mean_pinv.mean()),
                "ei_fbp_mean": float(e_fbp.mean()), "skei_fbp_mean": float(mean_fbp.mean()),
            })
        out["sketches"].append(item)
    return out
