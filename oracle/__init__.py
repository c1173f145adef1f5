"""FP64 CPU oracle for the sketched Equivariant Imaging hot path.

TEST INFRASTRUCTURE ONLY: imported by tests/, by ``__graft_entry__.smoke()``
and by the benchmark's CPU-baseline / reference leg, never by the product
package.  It shares no code with the CUDA library; the primitive operators
live in ``skei_oracle.c`` (plain loops), and this module composes them into
the paper's quantities with numpy in float64.

Paper map:
  * Sec. 2.1       y ~ A x, reconstruction F_theta(A^dagger y), A^dagger = FBP
  * Sec. 2.2, Eq. (e:eiloss)      EI loss = MC + lambda * EI regulariser
  * Sec. 3.1, Eq. (e:skeiloss)    sketched loss: A -> A_S = S A, y -> S y,
                                  A^dagger -> A_S^dagger
  * Sec. 3.2, Eq. (e:skeilossttt) the test-time (single measurement) form
  * Algorithm 2   per iteration: draw S_k and T_i, MC + lambda SkEI, Adam step
  * Sec. 4.2.1    CT sketch = one of N interleaved angle subsets
  * Sec. 4.1.3    transforms = rotations; Adam with lr 5e-4
  * Sec. 3.3      BN-only test-time training: batch-statistics BN layers,
                  only their affine parameters adapted
  * Algorithm 1   several measurements per step, a sketch drawn for each
  * Theorem 1     ||U^T (S^T S - I) U|| of the interleaved sketches of A
  * Sec. 3.4, Eq. (e:mri), Algorithm 3   multi-coil MRI A = M F C, PCA coil
                  compression and the coil sketch S_c = [I_R 0; 0 S_low]

Readings where the paper is silent (all recorded in the design notes):
  A_S^dagger is the FBP over the sketch's angles, (pi/m) B_S H; the sketch is
  an unscaled row selection, with the sketched MC term multiplied by
  ``mc_scale``; norms are sums of squares; loss = (1/B) sum_b
  [mc_b + lambda/G sum_g ei_bg]; a BN layer normalises with the biased batch
  variance plus eps = 1e-5.

Parity status: every function here is pinned by tests/test_oracle_*.py
(closed forms, exact symmetries, explicit small matrices, analytic Radon and
FBP convergence, finite differences, torch's Adam); none is "parity unpinned"
except the noise model of the inputs module, which is not part of the oracle.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "skei_oracle.c")
_LIB_DIR = os.path.join(_HERE, "_build")
_LIB = os.path.join(_LIB_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (FP contraction off, so x86 and Arm
    round identically)."""
    os.makedirs(_LIB_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
               "-fno-fast-math", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            D = ctypes.POINTER(ctypes.c_double)
            I = ctypes.c_int
            lib.oracle_ndet.argtypes = [I]
            lib.oracle_ndet.restype = I
            lib.oracle_trig.argtypes = [ctypes.c_double, D, D]
            lib.oracle_row_mode.argtypes = [ctypes.c_double]
            lib.oracle_row_mode.restype = I
            lib.oracle_ramlak_tap.argtypes = [I]
            lib.oracle_ramlak_tap.restype = ctypes.c_double
            for name in ("oracle_joseph_fwd", "oracle_joseph_adj",
                         "oracle_backproject", "oracle_backproject_adj"):
                getattr(lib, name).argtypes = [I, I, I, D, D, D]
            lib.oracle_ramlak.argtypes = [I, I, D, D]
            lib.oracle_rotate.argtypes = [I, ctypes.c_double, D, D]
            lib.oracle_rotate_adj.argtypes = [I, ctypes.c_double, D, D]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


# --------------------------------------------------------------------------
# geometry
# --------------------------------------------------------------------------

def ndet(N: int) -> int:
    """Detector bins: smallest odd integer >= N sqrt(2)."""
    return _load().oracle_ndet(int(N))


def trig(deg: float):
    c, s = ctypes.c_double(), ctypes.c_double()
    _load().oracle_trig(float(deg), ctypes.byref(c), ctypes.byref(s))
    return c.value, s.value


def row_mode(deg: float) -> bool:
    return bool(_load().oracle_row_mode(float(deg)))


def ramlak_tap(n: int) -> float:
    return _load().oracle_ramlak_tap(int(n))


# --------------------------------------------------------------------------
# primitive operators (batched over leading dims)
# --------------------------------------------------------------------------

def proj_fwd(x, angles_deg, n_det: int) -> np.ndarray:
    """A x: [..., N, N] -> [..., n_angles, n_det] (Joseph, Sec. 4.1.1)."""
    x = _f64(x)
    ang = _f64(angles_deg).ravel()
    N = x.shape[-1]
    lead = x.shape[:-2]
    xs = x.reshape(-1, N, N)
    out = np.empty((xs.shape[0], ang.size, n_det))
    for b in range(xs.shape[0]):
        xb = np.ascontiguousarray(xs[b])
        ob = np.empty((ang.size, n_det))
        _load().oracle_joseph_fwd(N, n_det, ang.size, _ptr(ang), _ptr(xb), _ptr(ob))
        out[b] = ob
    return out.reshape(lead + (ang.size, n_det))


def proj_adj(p, angles_deg, N: int) -> np.ndarray:
    """A^T p: [..., n_angles, n_det] -> [..., N, N] (scatter)."""
    p = _f64(p)
    ang = _f64(angles_deg).ravel()
    n_det = p.shape[-1]
    lead = p.shape[:-2]
    ps = p.reshape(-1, ang.size, n_det)
    out = np.empty((ps.shape[0], N, N))
    for b in range(ps.shape[0]):
        pb = np.ascontiguousarray(ps[b])
        ob = np.empty((N, N))
        _load().oracle_joseph_adj(N, n_det, ang.size, _ptr(ang), _ptr(pb), _ptr(ob))
        out[b] = ob
    return out.reshape(lead + (N, N))


def ramlak(p) -> np.ndarray:
    """H p, row by row: [..., n_det] -> [..., n_det]."""
    p = _f64(p)
    n_det = p.shape[-1]
    rows = int(np.prod(p.shape[:-1])) if p.ndim > 1 else 1
    q = np.empty_like(p)
    _load().oracle_ramlak(n_det, rows, _ptr(p), _ptr(q))
    return q


def backproject(q, angles_deg, N: int) -> np.ndarray:
    """B q (unscaled): [..., n_angles, n_det] -> [..., N, N]."""
    q = _f64(q)
    ang = _f64(angles_deg).ravel()
    n_det = q.shape[-1]
    lead = q.shape[:-2]
    qs = q.reshape(-1, ang.size, n_det)
    out = np.empty((qs.shape[0], N, N))
    for b in range(qs.shape[0]):
        qb = np.ascontiguousarray(qs[b])
        ob = np.empty((N, N))
        _load().oracle_backproject(N, n_det, ang.size, _ptr(ang), _ptr(qb), _ptr(ob))
        out[b] = ob
    return out.reshape(lead + (N, N))


def backproject_adj(x, angles_deg, n_det: int) -> np.ndarray:
    """B^T x (scatter): [..., N, N] -> [..., n_angles, n_det]."""
    x = _f64(x)
    ang = _f64(angles_deg).ravel()
    N = x.shape[-1]
    lead = x.shape[:-2]
    xs = x.reshape(-1, N, N)
    out = np.empty((xs.shape[0], ang.size, n_det))
    for b in range(xs.shape[0]):
        xb = np.ascontiguousarray(xs[b])
        ob = np.empty((ang.size, n_det))
        _load().oracle_backproject_adj(N, n_det, ang.size, _ptr(ang), _ptr(xb), _ptr(ob))
        out[b] = ob
    return out.reshape(lead + (ang.size, n_det))


def fbp(p, angles_deg, N: int) -> np.ndarray:
    """A^dagger p = (pi/m') B H p, m' = number of angles (Sec. 2.1: FBP as the
    stable approximation of the pseudo-inverse)."""
    ang = _f64(angles_deg).ravel()
    return (np.pi / ang.size) * backproject(ramlak(p), ang, N)


def fbp_adj(x, angles_deg, n_det: int) -> np.ndarray:
    """(A^dagger)^T x = (pi/m') H B^T x (H is symmetric)."""
    ang = _f64(angles_deg).ravel()
    return (np.pi / ang.size) * ramlak(backproject_adj(x, ang, n_det))


def rotate(x, g_deg: float) -> np.ndarray:
    """T_g x for one image [N, N]."""
    x = _f64(x)
    N = x.shape[-1]
    out = np.empty((N, N))
    _load().oracle_rotate(N, float(g_deg), _ptr(x), _ptr(out))
    return out


def rotate_adj(gout, g_deg: float) -> np.ndarray:
    gout = _f64(gout)
    N = gout.shape[-1]
    out = np.empty((N, N))
    _load().oracle_rotate_adj(N, float(g_deg), _ptr(gout), _ptr(out))
    return out


def rotate_batch(x, g_deg) -> np.ndarray:
    """x [B, N, N], g_deg [B, G] -> [B, G, N, N]."""
    x = _f64(x)
    g = np.asarray(g_deg, dtype=np.float64)
    B, G = g.shape
    return np.stack([np.stack([rotate(x[b], g[b, k]) for k in range(G)]) for b in range(B)])


def rotate_adj_batch(gout, g_deg) -> np.ndarray:
    """sum_g T_g^T gout[b, g]: [B, G, N, N] -> [B, N, N]."""
    gout = _f64(gout)
    g = np.asarray(g_deg, dtype=np.float64)
    B, G = g.shape
    return np.stack([sum(rotate_adj(gout[b, k], g[b, k]) for k in range(G)) for b in range(B)])


# --------------------------------------------------------------------------
# sketch (Sec. 3.1 and 4.2.1)
# --------------------------------------------------------------------------

def select(angles_deg, idx):
    """Angles of the sketch S: the rows of A kept by the selection."""
    ang = _f64(angles_deg).ravel()
    if idx is None:
        return ang
    return ang[np.asarray(idx, dtype=np.int64)]


# --------------------------------------------------------------------------
# EI / SkEI loss, split around the network F (Eq. e:skeiloss, Algorithm 2)
# --------------------------------------------------------------------------

def ei_stage1(x1, y, angles_deg, mc_idx, sk_idx, g_deg):
    """Everything the loss needs before the second network call.

    x1 = F(A^dagger y) [B, N, N]; y [B, n_angles, n_det].
    Returns r = S y - A_S x1 (MC residual, [B, m_mc, n_det]),
    x2 = T_g x1 ([B, G, N, N]) and z = A_S^dagger A_S x2 ([B, G, N, N])."""
    x1 = _f64(x1)
    y = _f64(y)
    N = x1.shape[-1]
    n_det = y.shape[-1]
    ang_mc = select(angles_deg, mc_idx)
    ang_sk = select(angles_deg, sk_idx)
    y_mc = y if mc_idx is None else y[:, np.asarray(mc_idx, dtype=np.int64), :]
    r = y_mc - proj_fwd(x1, ang_mc, n_det)
    x2 = rotate_batch(x1, g_deg)
    z = fbp(proj_fwd(x2, ang_sk, n_det), ang_sk, N)
    return r, x2, z


def ei_finish(x2, x3, r, lam: float, mc_scale: float):
    """mc_b = mc_scale ||r_b||^2, ei_bg = ||x2 - x3||^2,
    L = (1/B) sum_b [mc_b + (lambda/G) sum_g ei_bg]; also the seeds
    dL/dx2 = 2 lambda/(B G) (x2 - x3) = -dL/dx3."""
    x2, x3, r = _f64(x2), _f64(x3), _f64(r)
    B, G = x2.shape[:2]
    mc = mc_scale * np.sum(r.reshape(B, -1) ** 2, axis=1)
    d = x2 - x3
    ei = np.sum(d.reshape(B, G, -1) ** 2, axis=2)
    loss = float(np.mean(mc + (lam / G) * np.sum(ei, axis=1)))
    g_x2 = (2.0 * lam / (B * G)) * d
    return loss, mc, ei, g_x2, -g_x2


def ei_backward(r, g_x2, g_z, angles_deg, mc_idx, sk_idx, g_deg, mc_scale: float):
    """dL/dx1 = -(2 mc_scale / B) A_S^T r
               + sum_g T_g^T [g_x2 + (pi/m) A_S^T H B_S^T g_z]."""
    r, g_x2, g_z = _f64(r), _f64(g_x2), _f64(g_z)
    B, G, N = g_x2.shape[0], g_x2.shape[1], g_x2.shape[-1]
    n_det = r.shape[-1]
    ang_mc = select(angles_deg, mc_idx)
    ang_sk = select(angles_deg, sk_idx)
    g_tot = g_x2 + proj_adj(fbp_adj(g_z, ang_sk, n_det), ang_sk, N)
    return -(2.0 * mc_scale / B) * proj_adj(r, ang_mc, N) + rotate_adj_batch(g_tot, g_deg)


def ei_stage1_per_sample(x1, y, angles_deg, mc_rows, sk_rows, g_deg):
    """Algorithm 1 with a sketch drawn per measurement: measurement b uses row
    b of mc_rows / sk_rows ([B][m]; None = all angles) for its MC term and for
    the EI term of its transformed images.  Returns (r, x2, z) stacked over
    the measurements."""
    x1, y = _f64(x1), _f64(y)
    g = np.asarray(g_deg, dtype=np.float64)
    outs = [ei_stage1(x1[b:b + 1], y[b:b + 1], angles_deg,
                      None if mc_rows is None else mc_rows[b],
                      None if sk_rows is None else sk_rows[b], g[b:b + 1])
            for b in range(x1.shape[0])]
    return tuple(np.concatenate([o[i] for o in outs]) for i in range(3))


def ei_backward_per_sample(r, g_x2, g_z, angles_deg, mc_rows, sk_rows, g_deg,
                           mc_scale: float):
    """dL/dx1 for ei_stage1_per_sample.  The loss is the mean over the B
    measurements, so measurement b's MC term carries mc_scale / B
    (ei_backward of a single measurement applies 2 mc_scale)."""
    r, g_x2, g_z = _f64(r), _f64(g_x2), _f64(g_z)
    g = np.asarray(g_deg, dtype=np.float64)
    B = r.shape[0]
    return np.concatenate([
        ei_backward(r[b:b + 1], g_x2[b:b + 1], g_z[b:b + 1], angles_deg,
                    None if mc_rows is None else mc_rows[b],
                    None if sk_rows is None else sk_rows[b], g[b:b + 1], mc_scale / B)
        for b in range(B)])


# --------------------------------------------------------------------------
# stand-in network F_theta(u) = u + theta and the full test-time objective
# --------------------------------------------------------------------------

def ttt_loss(theta, x0, y, angles_deg, mc_idx, sk_idx, g_deg, lam, mc_scale):
    """Loss of Eq. (e:skeilossttt) (batched over B measurements) with the
    residual stand-in F(u) = u + theta (theta [N, N], shared by all b)."""
    x1 = _f64(x0) + _f64(theta)[None]
    r, x2, z = ei_stage1(x1, y, angles_deg, mc_idx, sk_idx, g_deg)
    x3 = z + _f64(theta)[None, None]
    loss, mc, ei, g_x2, g_x3 = ei_finish(x2, x3, r, lam, mc_scale)
    return loss, dict(r=r, x2=x2, z=z, x3=x3, mc=mc, ei=ei, g_x2=g_x2, g_x3=g_x3)


def ttt_grad(theta, x0, y, angles_deg, mc_idx, sk_idx, g_deg, lam, mc_scale):
    """(loss, dL/dtheta) for F(u) = u + theta: the chain rule through both
    network calls gives dL/dtheta = sum_b dL/dx1_b + sum_{b,g} dL/dx3_bg."""
    loss, t = ttt_loss(theta, x0, y, angles_deg, mc_idx, sk_idx, g_deg, lam, mc_scale)
    g_x1 = ei_backward(t["r"], t["g_x2"], t["g_x3"], angles_deg, mc_idx, sk_idx,
                       g_deg, mc_scale)
    return loss, g_x1.sum(axis=0) + t["g_x3"].sum(axis=(0, 1)), t


def ttt_loss_per_sample(theta, x0, y, angles_deg, mc_rows, sk_rows, g_deg, lam, mc_scale):
    """ttt_loss with a sketch per measurement (rows of mc_rows / sk_rows)."""
    x1 = _f64(x0) + _f64(theta)[None]
    r, x2, z = ei_stage1_per_sample(x1, y, angles_deg, mc_rows, sk_rows, g_deg)
    x3 = z + _f64(theta)[None, None]
    loss, mc, ei, g_x2, g_x3 = ei_finish(x2, x3, r, lam, mc_scale)
    return loss, dict(r=r, x2=x2, z=z, x3=x3, mc=mc, ei=ei, g_x2=g_x2, g_x3=g_x3)


def ttt_grad_per_sample(theta, x0, y, angles_deg, mc_rows, sk_rows, g_deg, lam, mc_scale):
    """(loss, dL/dtheta) of ttt_loss_per_sample."""
    loss, t = ttt_loss_per_sample(theta, x0, y, angles_deg, mc_rows, sk_rows, g_deg, lam,
                                  mc_scale)
    g_x1 = ei_backward_per_sample(t["r"], t["g_x2"], t["g_x3"], angles_deg, mc_rows, sk_rows,
                                  g_deg, mc_scale)
    return loss, g_x1.sum(axis=0) + t["g_x3"].sum(axis=(0, 1)), t


def adam_step(theta, grad, m, v, step: int, lr=5e-4, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma and Ba 2015), the optimiser of Algorithm 2 with
    the paper's lr 5e-4 (Sec. 4.1.3).  step counts from 1.  Returns new
    (theta, m, v)."""
    theta, grad, m, v = _f64(theta), _f64(grad), _f64(m), _f64(v)
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    m_hat = m / (1.0 - beta1 ** step)
    v_hat = v / (1.0 - beta2 ** step)
    return theta - lr * m_hat / (np.sqrt(v_hat) + eps), m, v


# --------------------------------------------------------------------------
# BN-only test-time training (Sec. 3.3): batch-statistics BN layers and the
# residual CNN stand-in built from them
# --------------------------------------------------------------------------

def _bn_parts(v, scale, shift, eps):
    axes = (0,) + tuple(range(2, v.ndim))
    shp = (1, -1) + (1,) * (v.ndim - 2)
    mu = v.mean(axis=axes, keepdims=True)
    var = ((v - mu) ** 2).mean(axis=axes, keepdims=True)
    sigma = np.sqrt(var + eps)
    xh = (v - mu) / sigma
    y = _f64(scale).reshape(shp) * xh + _f64(shift).reshape(shp)
    return axes, shp, sigma, xh, y


def bn_act(v, scale, shift, relu=True, eps=1e-5):
    """Sec. 3.3: BN(v) = theta_1 (v - mu) / sigma + theta_2 per channel of
    v [B, C, ...], mu and sigma the mean and standard deviation of the current
    batch (biased variance plus eps: the paper leaves both open), then ReLU."""
    v = _f64(v)
    _, _, _, _, y = _bn_parts(v, scale, shift, eps)
    return np.maximum(y, 0.0) if relu else y


def bn_act_bwd(v, g, scale, shift, relu=True, eps=1e-5):
    """Gradients of bn_act at v for the output gradient g, by the chain rule
    through the batch statistics: with g_y = g where the ReLU passes,
    d/dshift = sum g_y, d/dscale = sum g_y x^, and
    d/dv = (scale / sigma) (g_y - mean(g_y) - x^ mean(g_y x^))."""
    v, g = _f64(v), _f64(g)
    axes, shp, sigma, xh, y = _bn_parts(v, scale, shift, eps)
    gy = g * (y > 0) if relu else g
    g_shift = gy.sum(axis=axes)
    g_scale = (gy * xh).sum(axis=axes)
    M = v.size // v.shape[1]
    g_v = (_f64(scale).reshape(shp) / sigma) * (
        gy - g_shift.reshape(shp) / M - xh * g_scale.reshape(shp) / M)
    return g_v, g_scale, g_shift


def rescnn(u, conv, bn, eps=1e-5):
    """The residual CNN stand-in F(u) = u + h(u): h = 3x3 convolutions (zero
    padding 1, no bias), each but the last followed by bn_act with ReLU;
    u [n, N, N] (each image one batch entry, one channel); bn = the flat
    per-layer (scale, shift) vector.  Convolutions by torch's CPU conv2d in
    float64 (a library primitive)."""
    import torch
    import torch.nn.functional as tf
    u = _f64(u)
    h = u[:, None]
    C = conv[0].shape[0]
    for l, w in enumerate(conv):
        h = tf.conv2d(torch.from_numpy(h), torch.from_numpy(_f64(w)), padding=1).numpy()
        if l < len(conv) - 1:
            o = 2 * C * l
            h = bn_act(h, bn[o:o + C], bn[o + C:o + 2 * C], True, eps)
    return u + h[:, 0]


def ttt_bn_loss(bn, conv, x0, y, angles_deg, mc_idx, sk_idx, g_deg, lam, mc_scale, eps=1e-5):
    """Loss of Eq. (e:skeilossttt) with F = rescnn: x1 = F(x0) (the B
    measurements' A^dagger y as one batch), x3 = F(z) (the B G transformed
    reconstructions as one batch), as a function of the BN parameters."""
    x1 = rescnn(x0, conv, bn, eps)
    r, x2, z = ei_stage1(x1, y, angles_deg, mc_idx, sk_idx, g_deg)
    B, G, N = z.shape[0], z.shape[1], z.shape[-1]
    x3 = rescnn(z.reshape(B * G, N, N), conv, bn, eps).reshape(B, G, N, N)
    return ei_finish(x2, x3, r, lam, mc_scale)[0]


# --------------------------------------------------------------------------
# Theorem 1 (approximation bound of the sketched EI regulariser)
# --------------------------------------------------------------------------

def explicit_matrix(N: int, angles_deg, n_det: int) -> np.ndarray:
    """Joseph's A as a dense [len(angles) n_det, N^2] matrix, column j = A e_j."""
    d = N * N
    return proj_fwd(np.eye(d).reshape(d, N, N), angles_deg, n_det).reshape(d, -1).T.copy()


def sketch_gram_deviation(A, n_angles: int, n_det: int, ns: int, rank_tol: float = 1e-10):
    """||U^T (S^T S - I) U||_2 for each of the ns interleaved sketches of an
    n_angles-angle sinogram (offset o selects angles o, o + ns, ...), with
    S^T S = ns P_o (unbiased over the offsets) and U the left singular
    vectors of A for its singular values above rank_tol s_1 (the proof of
    Theorem 1).  Returns (deltas [ns], singular values kept)."""
    U, s, _ = np.linalg.svd(_f64(A), full_matrices=False)
    k = int(np.sum(s > rank_tol * s[0]))
    U = U[:, :k]
    out = []
    for o in range(ns):
        mask = np.zeros(n_angles)
        mask[o::ns] = 1.0
        rows = np.repeat(mask, n_det) > 0
        M = ns * (U[rows].T @ U[rows]) - np.eye(k)
        out.append(float(np.max(np.abs(np.linalg.eigvalsh(M)))))
    return np.array(out), s[:k]


# --------------------------------------------------------------------------
# multi-coil MRI (Sec. 3.4, Eq. (e:mri)) and the coil sketch (Algorithm 3)
# --------------------------------------------------------------------------

def _cplx(a):
    a = _f64(a)
    return a[..., 0, :, :] + 1j * a[..., 1, :, :]


def _planar(z):
    return np.stack([z.real, z.imag], axis=-3)


def mri_fwd(x, maps, mask=None):
    """Eq. (e:mri): k_c = M F (C_c x), F the unitary 2D DFT (frequency 0 at
    index 0).  x planar [B, 2, N, N], maps [Nc, 2, N, N] -> [B, Nc, 2, N, N].
    The DFT is numpy's fft2 (a library primitive, norm "ortho")."""
    k = np.fft.fft2(_cplx(maps)[None] * _cplx(x)[:, None], norm="ortho")
    if mask is not None:
        k = k * _f64(mask)
    return _planar(k)


def mri_adj(k, maps, mask=None):
    """A^H k = sum_c conj(C_c) F^H (M k_c): [B, Nc, 2, N, N] -> [B, 2, N, N]."""
    kc = _cplx(k)
    if mask is not None:
        kc = kc * _f64(mask)
    return _planar(np.sum(np.conj(_cplx(maps))[None] * np.fft.ifft2(kc, norm="ortho"), axis=1))


def mri_dinv(maps):
    """1 / sum_c |C_c|^2 per pixel, 0 where the sum is 0."""
    s = np.sum(np.abs(_cplx(maps)) ** 2, axis=0)
    out = np.zeros_like(s)
    out[s > 0] = 1.0 / s[s > 0]
    return out


def mri_pinv(k, maps, mask=None):
    """A^dagger k = dinv A^H k: the coil-combined zero-filled inverse (the
    least-squares inverse of F C when every sample is taken)."""
    return mri_adj(k, maps, mask) * mri_dinv(maps)[None, None]


def coil_mix(W, x):
    """out[b, j] = sum_i W[j, i] x[b, i] for complex W [n_out, n_in] and
    planar coil data x [B, n_in, 2, ...]."""
    return _planar(np.einsum("ji,bi...->bj...", np.asarray(W, dtype=np.complex128), _cplx(x)))


def coil_pca(k, L: int):
    """Algorithm 3 / Sec. 3.4's PCA coil compression of one measurement's
    k-space k [Nc, 2, N, N]: centre each coil over its d samples, covariance
    V_ij = conj(kbar_i) . kbar_j / (d - 1), and the L dominant eigenvectors
    Q_L [Nc, L] (eigenvalues descending; each eigenvector's phase fixed so
    that its largest-magnitude entry, the first such, is real positive).
    Virtual coil l is sum_c Q[c, l] k_c."""
    K = _cplx(k).reshape(k.shape[0], -1).T                    # [d, Nc]
    Kb = K - K.mean(axis=0, keepdims=True)
    V = Kb.conj().T @ Kb / (K.shape[0] - 1)
    w, Q = np.linalg.eigh(V)
    order = np.argsort(-w, kind="stable")
    Q = Q[:, order][:, :L]
    for l in range(L):
        i = int(np.argmax(np.abs(Q[:, l])))
        Q[:, l] *= np.conj(Q[i, l]) / abs(Q[i, l])
    return Q, w[order]


def coil_sketch(L: int, R: int, s_low):
    """S_c = [[I_R, 0], [0, S_low]] [M_c, L] of Sec. 3.4, S_low the
    (M_c - R) x (L - R) Rademacher block."""
    s_low = np.asarray(s_low, dtype=np.float64)
    Mc = R + s_low.shape[0]
    S = np.zeros((Mc, L))
    S[:R, :R] = np.eye(R)
    S[R:, R:] = s_low
    return S


def mri_ttt_loss(theta, x0, y, maps, mask, g_deg, lam):
    """Sec. 3.4's coil-sketched EI loss for one measurement with the residual
    stand-in F(u) = u + theta (theta planar [2, N, N]): MC ||y - A x1||^2 and
    EI (lambda/G) sum_g ||T_g x1 - F(A^dagger A T_g x1)||^2, A = (maps, mask)
    (the sketched maps and data for C-SkEI); T_g rotates both planes."""
    x1 = _f64(x0) + _f64(theta)[None]
    r = _f64(y) - mri_fwd(x1, maps, mask)
    G = np.asarray(g_deg).shape[1]
    x2 = np.stack([np.stack([rotate(x1[0, c], g_deg[0][g]) for c in range(2)])
                   for g in range(G)])[None]                    # [1, G, 2, N, N]
    z = mri_pinv(mri_fwd(x2[0], maps, mask), maps, mask)[None]
    x3 = z + _f64(theta)[None, None]
    loss, mc, ei, g_x2, g_x3 = ei_finish(x2, x3, r, lam, 1.0)
    return loss, dict(r=r, x2=x2, z=z, x3=x3, g_x2=g_x2, g_x3=g_x3)


def mri_ttt_grad(theta, x0, y, maps, mask, g_deg, lam):
    """(loss, dL/dtheta) of mri_ttt_loss: the planar real gradient of a
    complex-linear map P is its adjoint P^H, and (A^dagger A)^H = A^H A dinv,
    so dL/dx1 = -2 A^H r + sum_g T_g^T [g_x2 + A^H A (dinv g_z)]."""
    loss, t = mri_ttt_loss(theta, x0, y, maps, mask, g_deg, lam)
    G = t["x2"].shape[1]
    dinv = mri_dinv(maps)
    g_z = t["g_x3"][0]                                          # [G, 2, N, N]
    g_tot = t["g_x2"][0] + mri_adj(mri_fwd(g_z * dinv[None, None], maps, mask), maps, mask)
    g_x1 = -2.0 * mri_adj(t["r"], maps, mask)[0]
    for g in range(G):
        for c in range(2):
            g_x1[c] += rotate_adj(g_tot[g, c], g_deg[0][g])
    return loss, g_x1 + t["g_x3"][0].sum(axis=0), t


def psnr(x, ref) -> float:
    """10 log10(range^2 / MSE), range = max(ref) - min(ref)."""
    x, ref = _f64(x), _f64(ref)
    mse = float(np.mean((x - ref) ** 2))
    rng = float(ref.max() - ref.min())
    return 10.0 * np.log10(rng * rng / mse)
