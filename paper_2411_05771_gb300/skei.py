"""Thin Python binding of libskei (include/skei.h).

Every function here marshals torch tensors into the C ABI of the same name
(``proj_fwd`` -> ``skei_proj_fwd`` and so on) and launches on the current
torch CUDA stream; all arithmetic runs in the library's CUDA kernels.  There
is no fallback: importing this module fails if libskei.so is missing, and
every call fails on non-CUDA tensors.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

from . import build as _build

__all__ = [
    "F32", "BF16", "Plan", "last_error", "version",
    "proj_fwd", "proj_adj", "proj_fwd_multi", "proj_adj_multi", "Job",
    "band_sums_workspace_size", "proj_fwd_multi_ws", "backproject_adj_multi_ws",
    "filter", "filter_fft", "filter_tc", "backproject", "backproject_adj",
    "fbp_workspace_size", "fbp", "fbp_adj", "fbp_noalloc", "rotate", "rotate_adj",
    "ei_workspace_size", "ei_fwd_form", "ei_loss_fwd", "ei_loss_finish", "ei_loss_bwd",
    "ei_loss_fwd_per_sample", "ei_loss_bwd_per_sample",
    "residual_add", "adam_step", "step_draws", "library_path",
    "bn_workspace_size", "bn_act_fwd", "bn_act_bwd",
    "mri_workspace_size", "mri_fwd", "mri_adj", "mri_dinv", "coil_mix",
    "Batch", "BatchItem", "PROJ_FWD", "PROJ_ADJ", "BACKPROJECT", "BACKPROJECT_ADJ", "FILTER",
    "FBP", "measure_roofs", "ROOFS_WORK_BYTES", "ttt_residual_workspace_size", "check_build",
    "check_status",
    "ttt_residual_step",
]

F32, BF16 = 0, 1
ROOFS_WORK_BYTES = 1 << 30

# SKEI_LIBRARY selects another build of the same library (the bounds-check
# build, libskei_check.so)
library_path = os.environ.get("SKEI_LIBRARY") or _build.LIB
if not os.path.exists(library_path):
    raise ImportError(
        f"libskei.so not found at {library_path}; build it with "
        "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc)")
_lib = ctypes.CDLL(library_path)

_vp, _i, _f, _d, _sz, _i64 = (ctypes.c_void_p, ctypes.c_int, ctypes.c_float, ctypes.c_double,
                              ctypes.c_size_t, ctypes.c_int64)
_PLAN = ctypes.c_void_p


class _Job(ctypes.Structure):
    _fields_ = [("dtype_in", ctypes.c_int), ("dtype_aux", ctypes.c_int),
                ("dtype_out", ctypes.c_int), ("in_", ctypes.c_void_p), ("aux", ctypes.c_void_p),
                ("out", ctypes.c_void_p), ("idx", ctypes.c_void_p), ("m", ctypes.c_int),
                ("B", ctypes.c_int), ("alpha", ctypes.c_float), ("beta", ctypes.c_float)]


class _Roofs(ctypes.Structure):
    _fields_ = [("fp32_flops", ctypes.c_double), ("smem_bytes", ctypes.c_double),
                ("l2_bytes", ctypes.c_double), ("dram_read_bytes", ctypes.c_double),
                ("sms", ctypes.c_int)]


class _BatchItemC(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("dtype_in", ctypes.c_int),
                ("dtype_out", ctypes.c_int), ("in_", ctypes.c_void_p), ("out", ctypes.c_void_p),
                ("idx", ctypes.c_void_p), ("m", ctypes.c_int), ("B", ctypes.c_int),
                ("scale", ctypes.c_float)]


_BATCH = ctypes.c_void_p

_SIGS = {
    "skei_version": ([], _i),
    "skei_last_error": ([], ctypes.c_char_p),
    "skei_plan_create": ([_i, _i, _i, _vp, ctypes.POINTER(_PLAN)], _i),
    "skei_plan_destroy": ([_PLAN], _i),
    "skei_plan_geometry": ([_PLAN, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i)], _i),
    "skei_plan_status": ([_PLAN, _i, ctypes.POINTER(_i)], _i),
    "skei_proj_fwd": ([_PLAN, _i, _vp, _i, _vp, _i, _vp, _vp, _vp], _i),
    "skei_proj_adj": ([_PLAN, _i, _vp, _i, _vp, _i, _f, _f, _vp, _vp], _i),
    "skei_filter": ([_PLAN, _i, _vp, _i, _f, _vp, _vp], _i),
    "skei_filter_fft": ([_PLAN, _i, _vp, _i, _f, _vp, _vp], _i),
    "skei_filter_tc": ([_PLAN, _i, _vp, _i, _f, _vp, _vp], _i),
    "skei_proj_fwd_multi": ([_PLAN, ctypes.POINTER(_Job), _i, _vp], _i),
    "skei_proj_adj_multi": ([_PLAN, ctypes.POINTER(_Job), _i, _vp], _i),
    "skei_band_sums_workspace_size": ([_PLAN, ctypes.POINTER(_Job), _i], _sz),
    "skei_proj_fwd_multi_ws": ([_PLAN, ctypes.POINTER(_Job), _i, _vp, _sz, _vp], _i),
    "skei_backproject_adj_multi_ws": ([_PLAN, ctypes.POINTER(_Job), _i, _vp, _sz, _vp], _i),
    "skei_backproject": ([_PLAN, _i, _vp, _i, _vp, _i, _f, _f, _vp, _vp], _i),
    "skei_backproject_adj": ([_PLAN, _i, _vp, _i, _vp, _i, _f, _vp, _vp], _i),
    "skei_fbp_workspace_size": ([_PLAN, _i, _i, _i], _sz),
    "skei_fbp": ([_PLAN, _i, _vp, _i, _vp, _i, _vp, _vp, _sz, _vp], _i),
    "skei_fbp_adj": ([_PLAN, _i, _vp, _i, _vp, _i, _vp, _vp, _sz, _vp], _i),
    "skei_fbp_noalloc": ([_PLAN, _i, _vp, _i, _vp, _i, _vp, _vp], _i),
    "skei_rotate": ([_i, _vp, _i, _i, _vp, _i, _vp, _vp], _i),
    "skei_rotate_adj": ([_i, _vp, _i, _i, _vp, _i, _f, _f, _vp, _vp], _i),
    "skei_rotate_channels": ([_i, _vp, _i, _i, _i, _vp, _i, _vp, _vp], _i),
    "skei_rotate_adj_channels": ([_i, _vp, _i, _i, _i, _vp, _i, _f, _f, _vp, _vp], _i),
    "skei_ei_finish_len_workspace_size": ([_i, _i, _i64, _i], _sz),
    "skei_ei_loss_finish_len": ([_i, _vp, _vp, _vp, _i, _i, _i64, _i, _d, _d, _vp, _vp, _vp,
                                 _vp, _vp, _vp, _sz, _vp], _i),
    "skei_ei_workspace_size": ([_PLAN, _i, _i, _i, _i, _i], _sz),
    "skei_ei_fwd_form": ([_PLAN, _i, _i, _vp, _i, _vp, _i, _i], _i),
    "skei_ei_finish_workspace_size": ([_i, _i, _i, _i], _sz),
    "skei_ei_loss_fwd": ([_PLAN, _i, _vp, _vp, _i, _vp, _i, _vp, _i, _vp, _i, _vp, _vp, _vp,
                          _vp, _sz, _vp], _i),
    "skei_ei_loss_finish": ([_i, _vp, _vp, _vp, _i, _i, _i, _i, _d, _d, _vp, _vp, _vp, _vp,
                             _vp, _vp, _sz, _vp], _i),
    "skei_ei_loss_bwd": ([_PLAN, _i, _vp, _vp, _vp, _i, _vp, _i, _vp, _i, _vp, _i, _d, _vp,
                          _vp, _sz, _vp], _i),
    "skei_ei_loss_fwd_per_sample": ([_PLAN, _i, _vp, _vp, _i, _vp, _i, _vp, _i, _vp, _i, _vp, _vp,
                                     _vp, _vp, _sz, _vp], _i),
    "skei_ei_loss_bwd_per_sample": ([_PLAN, _i, _vp, _vp, _vp, _i, _vp, _i, _vp, _i, _vp, _i, _d,
                                     _vp, _vp, _sz, _vp], _i),
    "skei_residual_add": ([_i, _vp, _vp, _i, _i64, _vp, _vp], _i),
    "skei_adam_step": ([_vp, _i64, _i, _vp, _i, _vp, _i, _vp, _vp, _vp, _d, _d, _d, _d, _vp], _i),
    "skei_step_draws": ([_vp, _i, _i64, _vp, _vp, _vp], _i),
    "skei_bn_workspace_size": ([_i, _i, _i64], _sz),
    "skei_bn_act_fwd": ([_i, _vp, _i, _i, _i64, _vp, _vp, _i, _d, _vp, _vp, _vp, _vp, _sz, _vp],
                        _i),
    "skei_bn_act_bwd": ([_i, _vp, _vp, _i, _i, _i64, _vp, _vp, _vp, _vp, _i, _vp, _vp, _vp, _vp,
                         _sz, _vp], _i),
    "skei_mri_workspace_size": ([_i, _i, _i], _sz),
    "skei_mri_fwd": ([_i, _i, _i, _vp, _vp, _vp, _vp, _vp, _f, _vp, _vp, _sz, _vp], _i),
    "skei_mri_adj": ([_i, _i, _i, _vp, _vp, _vp, _vp, _f, _f, _vp, _vp, _sz, _vp], _i),
    "skei_mri_dinv": ([_i, _i, _vp, _vp, _vp], _i),
    "skei_coil_mix": ([_i, _i, _i, _i, _vp, _vp, _vp, _vp], _i),
    "skei_batch_create": ([_i, ctypes.POINTER(_BatchItemC), _i, ctypes.POINTER(_BATCH)], _i),
    "skei_batch_run": ([_BATCH, _vp], _i),
    "skei_batch_tune": ([_BATCH, _i, _vp], _i),
    "skei_batch_info": ([_BATCH, _i, ctypes.POINTER(_i), ctypes.POINTER(_i), ctypes.POINTER(_i),
                         ctypes.POINTER(_i)], _i),
    "skei_batch_destroy": ([_BATCH], _i),
    "skei_measure_roofs": ([_vp, _sz, ctypes.POINTER(_Roofs), _vp], _i),
    "skei_check_build": ([], _i),
    "skei_check_status": ([ctypes.POINTER(ctypes.c_uint), _i], _i),
    "skei_ttt_residual_workspace_size": ([_PLAN, _i, _i, _i, _i, _i], _sz),
    "skei_ttt_residual_step": ([_PLAN, _i, _vp, _vp, _vp, _vp, _vp, _vp, _i, _vp, _i, _vp, _i,
                                _vp, _i, _d, _d, _d, _d, _d, _d] + [_vp] * 11 + [_vp, _sz, _vp],
                               _i),
}
for _name, (_args, _res) in _SIGS.items():
    _fn = getattr(_lib, _name)
    _fn.argtypes = _args
    _fn.restype = _res


def last_error() -> str:
    return _lib.skei_last_error().decode()


def version() -> int:
    return _lib.skei_version()


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"{what} failed ({rc}): {last_error()}")


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _dtype_code(t: torch.Tensor) -> int:
    if t.dtype == torch.float32:
        return F32
    if t.dtype == torch.bfloat16:
        return BF16
    raise TypeError(f"unsupported dtype {t.dtype}: use float32 or bfloat16")


def _dev(t, name, dtype=None, shape=None):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    return ctypes.c_void_p(t.data_ptr())


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


class Plan:
    """Geometry of A: image side N, detector bins n_det (0 = smallest odd
    >= N sqrt 2) and the full angle list in degrees (default 180 a / n)."""

    def __init__(self, N: int, n_angles: int, angles_deg=None, n_det: int = 0):
        self._h = _PLAN()
        ang = None
        if angles_deg is not None:
            ang = np.ascontiguousarray(np.asarray(angles_deg, dtype=np.float64).ravel())
            if ang.size != n_angles:
                raise ValueError("angles_deg must hold n_angles values")
        p = None if ang is None else ang.ctypes.data_as(ctypes.c_void_p)
        _check(_lib.skei_plan_create(int(N), int(n_det), int(n_angles), p, ctypes.byref(self._h)),
               "skei_plan_create")
        n, d, a = _i(), _i(), _i()
        _check(_lib.skei_plan_geometry(self._h, ctypes.byref(n), ctypes.byref(d), ctypes.byref(a)),
               "skei_plan_geometry")
        self.N, self.n_det, self.n_angles = n.value, d.value, a.value
        self.angles_deg = (ang.copy() if ang is not None
                           else 180.0 * np.arange(n_angles, dtype=np.float64) / n_angles)

    @property
    def handle(self):
        if not self._h:
            raise RuntimeError("plan is closed")
        return self._h

    def status(self, reset: bool = True) -> int:
        w = _i()
        _check(_lib.skei_plan_status(self.handle, int(reset), ctypes.byref(w)), "skei_plan_status")
        return w.value

    def close(self):
        if self._h:
            _lib.skei_plan_destroy(self._h)
            self._h = _PLAN()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _idx(plan: Plan, idx):
    if idx is None:
        return None, plan.n_angles
    _dev(idx, "idx", torch.int32)
    return ctypes.c_void_p(idx.data_ptr()), int(idx.numel())


def proj_fwd(plan: Plan, x: torch.Tensor, idx=None, y=None, out=None) -> torch.Tensor:
    """A_S x (or S y - A_S x when y is given); x [B, N, N] -> [B, m, n_det]."""
    B = x.shape[0]
    ip, m = _idx(plan, idx)
    _dev(x, "x", shape=(B, plan.N, plan.N))
    if y is not None:
        _dev(y, "y", x.dtype, (B, plan.n_angles, plan.n_det))
    if out is None:
        out = torch.empty((B, m, plan.n_det), device=x.device, dtype=x.dtype)
    _dev(out, "out", x.dtype, (B, m, plan.n_det))
    _check(_lib.skei_proj_fwd(plan.handle, _dtype_code(x), _ptr(x), B, ip, m, _ptr(y), _ptr(out),
                              _stream()), "skei_proj_fwd")
    return out


def proj_adj(plan: Plan, sino, idx=None, alpha=1.0, beta=0.0, out=None) -> torch.Tensor:
    """alpha A_S^T sino + beta out; sino [B, m, n_det] -> [B, N, N]."""
    B = sino.shape[0]
    ip, m = _idx(plan, idx)
    _dev(sino, "sino", shape=(B, m, plan.n_det))
    if out is None:
        if beta != 0.0:
            raise ValueError("beta != 0 needs out")
        out = torch.empty((B, plan.N, plan.N), device=sino.device, dtype=sino.dtype)
    _dev(out, "out", sino.dtype, (B, plan.N, plan.N))
    _check(_lib.skei_proj_adj(plan.handle, _dtype_code(sino), _ptr(sino), B, ip, m, float(alpha),
                              float(beta), _ptr(out), _stream()), "skei_proj_adj")
    return out


class Job:
    """One image set of a batched projector launch (see skei_job)."""

    def __init__(self, inp, out, idx=None, aux=None, alpha=1.0, beta=0.0):
        self.inp, self.out, self.idx, self.aux = inp, out, idx, aux
        self.alpha, self.beta = alpha, beta


def _jobs(plan: Plan, jobs, fwd: bool):
    arr = (_Job * len(jobs))()
    for q, jb in enumerate(jobs):
        _dev(jb.inp, "job.inp")
        _dev(jb.out, "job.out")
        ip, m = _idx(plan, jb.idx)
        use_aux = jb.aux is not None
        if use_aux:
            _dev(jb.aux, "job.aux")
        B = jb.inp.shape[0]
        if fwd:
            if tuple(jb.inp.shape) != (B, plan.N, plan.N) or tuple(jb.out.shape) != (B, m, plan.n_det):
                raise ValueError("job shapes: in [B,N,N], out [B,m,n_det]")
        else:
            if tuple(jb.inp.shape) != (B, m, plan.n_det) or tuple(jb.out.shape) != (B, plan.N, plan.N):
                raise ValueError("job shapes: in [B,m,n_det], out [B,N,N]")
        arr[q] = _Job(_dtype_code(jb.inp), _dtype_code(jb.aux) if use_aux else 0,
                      _dtype_code(jb.out), jb.inp.data_ptr(),
                      jb.aux.data_ptr() if use_aux else None, jb.out.data_ptr(),
                      ip.value if ip is not None else None, m, B, float(jb.alpha), float(jb.beta))
    return arr


def proj_fwd_multi(plan: Plan, jobs) -> None:
    """Several A_S (or S y - A_S x) applications in one launch."""
    arr = _jobs(plan, jobs, True)
    _check(_lib.skei_proj_fwd_multi(plan.handle, arr, len(jobs), _stream()), "skei_proj_fwd_multi")


def proj_adj_multi(plan: Plan, jobs) -> None:
    """Several alpha A_S^T in + beta aux applications in one launch."""
    arr = _jobs(plan, jobs, False)
    _check(_lib.skei_proj_adj_multi(plan.handle, arr, len(jobs), _stream()), "skei_proj_adj_multi")


def band_sums_workspace_size(plan: Plan, jobs) -> int:
    """Bytes of workspace the *_multi_ws forms need for these jobs."""
    arr = _jobs(plan, jobs, True)
    return int(_lib.skei_band_sums_workspace_size(plan.handle, arr, len(jobs)))


def proj_fwd_multi_ws(plan: Plan, jobs, work=None) -> None:
    """proj_fwd_multi through per-band sums in a workspace (two launches)."""
    arr = _jobs(plan, jobs, True)
    nbytes = int(_lib.skei_band_sums_workspace_size(plan.handle, arr, len(jobs)))
    w = _work(nbytes, jobs[0].inp.device, work)
    _check(_lib.skei_proj_fwd_multi_ws(plan.handle, arr, len(jobs), _ptr(w),
                                       w.numel() * w.element_size(), _stream()),
           "skei_proj_fwd_multi_ws")


def backproject_adj_multi_ws(plan: Plan, jobs, work=None) -> None:
    """Several out = alpha B_S^T in (in [B,N,N], out [B,m,n_det]) through
    per-band sums in a workspace (two launches)."""
    arr = _jobs(plan, jobs, True)
    nbytes = int(_lib.skei_band_sums_workspace_size(plan.handle, arr, len(jobs)))
    w = _work(nbytes, jobs[0].inp.device, work)
    _check(_lib.skei_backproject_adj_multi_ws(plan.handle, arr, len(jobs), _ptr(w),
                                              w.numel() * w.element_size(), _stream()),
           "skei_backproject_adj_multi_ws")


def filter(plan: Plan, p, scale=1.0, out=None) -> torch.Tensor:  # noqa: A001
    """scale * H p along the last (detector) axis."""
    if p.shape[-1] != plan.n_det:
        raise ValueError("last axis must hold n_det bins")
    _dev(p, "p")
    out = torch.empty_like(p) if out is None else out
    _dev(out, "out", p.dtype, p.shape)
    rows = p.numel() // plan.n_det
    _check(_lib.skei_filter(plan.handle, _dtype_code(p), _ptr(p), rows, float(scale), _ptr(out),
                            _stream()), "skei_filter")
    return out


def filter_fft(plan: Plan, p, scale=1.0, out=None) -> torch.Tensor:
    """filter() through the FFT (equal up to FP32 rounding); out must not alias p."""
    if p.shape[-1] != plan.n_det:
        raise ValueError("last axis must hold n_det bins")
    _dev(p, "p")
    out = torch.empty_like(p) if out is None else out
    _dev(out, "out", p.dtype, p.shape)
    rows = p.numel() // plan.n_det
    _check(_lib.skei_filter_fft(plan.handle, _dtype_code(p), _ptr(p), rows, float(scale),
                                _ptr(out), _stream()), "skei_filter_fft")
    return out


def filter_tc(plan: Plan, p, scale=1.0, out=None) -> torch.Tensor:
    """filter() as tensor-core matrix products (equal up to FP32 rounding);
    out must not alias p."""
    if p.shape[-1] != plan.n_det:
        raise ValueError("last axis must hold n_det bins")
    _dev(p, "p")
    out = torch.empty_like(p) if out is None else out
    _dev(out, "out", p.dtype, p.shape)
    rows = p.numel() // plan.n_det
    _check(_lib.skei_filter_tc(plan.handle, _dtype_code(p), _ptr(p), rows, float(scale),
                               _ptr(out), _stream()), "skei_filter_tc")
    return out


def backproject(plan: Plan, q, idx=None, alpha=1.0, beta=0.0, out=None) -> torch.Tensor:
    B = q.shape[0]
    ip, m = _idx(plan, idx)
    _dev(q, "q", shape=(B, m, plan.n_det))
    if out is None:
        if beta != 0.0:
            raise ValueError("beta != 0 needs out")
        out = torch.empty((B, plan.N, plan.N), device=q.device, dtype=q.dtype)
    _dev(out, "out", q.dtype, (B, plan.N, plan.N))
    _check(_lib.skei_backproject(plan.handle, _dtype_code(q), _ptr(q), B, ip, m, float(alpha),
                                 float(beta), _ptr(out), _stream()), "skei_backproject")
    return out


def backproject_adj(plan: Plan, x, idx=None, alpha=1.0, out=None) -> torch.Tensor:
    B = x.shape[0]
    ip, m = _idx(plan, idx)
    _dev(x, "x", shape=(B, plan.N, plan.N))
    if out is None:
        out = torch.empty((B, m, plan.n_det), device=x.device, dtype=x.dtype)
    _dev(out, "out", x.dtype, (B, m, plan.n_det))
    _check(_lib.skei_backproject_adj(plan.handle, _dtype_code(x), _ptr(x), B, ip, m, float(alpha),
                                     _ptr(out), _stream()), "skei_backproject_adj")
    return out


def fbp_workspace_size(plan: Plan, dtype: int, B: int, m: int) -> int:
    return int(_lib.skei_fbp_workspace_size(plan.handle, dtype, B, m))


def _work(nbytes: int, device, work=None):
    if work is not None:
        if work.numel() * work.element_size() < nbytes:
            raise ValueError("workspace too small")
        return work
    return torch.empty(max(nbytes, 16), dtype=torch.uint8, device=device)


def fbp(plan: Plan, sino, idx=None, out=None, work=None) -> torch.Tensor:
    """A_S^dagger sino = (pi/m) B_S H sino; [B, m, n_det] -> [B, N, N]."""
    B = sino.shape[0]
    ip, m = _idx(plan, idx)
    _dev(sino, "sino", shape=(B, m, plan.n_det))
    out = torch.empty((B, plan.N, plan.N), device=sino.device, dtype=sino.dtype) if out is None else out
    _dev(out, "out", sino.dtype, (B, plan.N, plan.N))
    code = _dtype_code(sino)
    nb = fbp_workspace_size(plan, code, B, m)
    w = _work(nb, sino.device, work)
    _check(_lib.skei_fbp(plan.handle, code, _ptr(sino), B, ip, m, _ptr(out), _ptr(w), nb,
                         _stream()), "skei_fbp")
    return out


def fbp_adj(plan: Plan, x, idx=None, out=None, work=None) -> torch.Tensor:
    B = x.shape[0]
    ip, m = _idx(plan, idx)
    _dev(x, "x", shape=(B, plan.N, plan.N))
    out = torch.empty((B, m, plan.n_det), device=x.device, dtype=x.dtype) if out is None else out
    _dev(out, "out", x.dtype, (B, m, plan.n_det))
    code = _dtype_code(x)
    nb = fbp_workspace_size(plan, code, B, m)
    w = _work(nb, x.device, work)
    _check(_lib.skei_fbp_adj(plan.handle, code, _ptr(x), B, ip, m, _ptr(out), _ptr(w), nb,
                             _stream()), "skei_fbp_adj")
    return out


FBP_NOALLOC_MAX_FLOATS = 1048576


def fbp_noalloc(plan: Plan, sino, idx=None, out=None) -> torch.Tensor:
    """skei_fbp_noalloc: the FBP of `fbp` without a workspace, for callers
    that cannot allocate device memory (its scratch is a static 4 MiB array
    inside the library; B * m * n_det <= FBP_NOALLOC_MAX_FLOATS; calls that
    overlap on the GPU race on that array).  `out` must be given by a caller
    that allocates nothing."""
    B = sino.shape[0]
    ip, m = _idx(plan, idx)
    _dev(sino, "sino", shape=(B, m, plan.n_det))
    out = torch.empty((B, plan.N, plan.N), device=sino.device, dtype=sino.dtype) if out is None else out
    _dev(out, "out", sino.dtype, (B, plan.N, plan.N))
    _check(_lib.skei_fbp_noalloc(plan.handle, _dtype_code(sino), _ptr(sino), B, ip, m, _ptr(out),
                                 _stream()), "skei_fbp_noalloc")
    return out


def rotate(x, g_deg, out=None) -> torch.Tensor:
    """T_g x for every (b, g): x [B, N, N] -> [B, G, N, N], or x [B, Ch, N, N]
    (channels rotated alike) -> [B, G, Ch, N, N]; g_deg float64 [B, G]."""
    B, N = x.shape[0], x.shape[-1]
    G = g_deg.shape[1]
    Ch = x.shape[1] if x.dim() == 4 else 1
    shp_in = (B, Ch, N, N) if x.dim() == 4 else (B, N, N)
    shp_out = (B, G, Ch, N, N) if x.dim() == 4 else (B, G, N, N)
    _dev(x, "x", shape=shp_in)
    _dev(g_deg, "g_deg", torch.float64, (B, G))
    out = torch.empty(shp_out, device=x.device, dtype=x.dtype) if out is None else out
    _dev(out, "out", x.dtype, shp_out)
    _check(_lib.skei_rotate_channels(_dtype_code(x), _ptr(x), B, Ch, N, _ptr(g_deg), G,
                                     _ptr(out), _stream()), "skei_rotate_channels")
    return out


def rotate_adj(gout, g_deg, alpha=1.0, beta=0.0, out=None) -> torch.Tensor:
    """alpha sum_g T_g^T gout[:, g] + beta out: [B, G, N, N] -> [B, N, N], or
    [B, G, Ch, N, N] -> [B, Ch, N, N]."""
    B, G, N = gout.shape[0], gout.shape[1], gout.shape[-1]
    Ch = gout.shape[2] if gout.dim() == 5 else 1
    shp_in = (B, G, Ch, N, N) if gout.dim() == 5 else (B, G, N, N)
    shp_out = (B, Ch, N, N) if gout.dim() == 5 else (B, N, N)
    _dev(gout, "gout", shape=shp_in)
    _dev(g_deg, "g_deg", torch.float64, (B, G))
    if out is None:
        if beta != 0.0:
            raise ValueError("beta != 0 needs out")
        out = torch.empty(shp_out, device=gout.device, dtype=gout.dtype)
    _dev(out, "out", gout.dtype, shp_out)
    _check(_lib.skei_rotate_adj_channels(_dtype_code(gout), _ptr(gout), B, Ch, N, _ptr(g_deg), G,
                                         float(alpha), float(beta), _ptr(out), _stream()),
           "skei_rotate_adj_channels")
    return out


def ei_workspace_size(plan: Plan, dtype: int, B: int, G: int, mc_m: int, sk_m: int) -> int:
    return int(_lib.skei_ei_workspace_size(plan.handle, dtype, B, G, mc_m, sk_m))


def _idx_rows(plan: Plan, idx, B: int, per_sample: bool):
    if not per_sample:
        return _idx(plan, idx)
    if idx is None:
        return None, plan.n_angles
    _dev(idx, "idx", torch.int32)
    if idx.dim() != 2 or idx.shape[0] != B:
        raise ValueError(f"per-sample idx must be [B={B}, m], got {tuple(idx.shape)}")
    return ctypes.c_void_p(idx.data_ptr()), int(idx.shape[1])


def ei_fwd_form(plan: Plan, B: int, G: int, mc_idx=None, sk_idx=None,
                per_sample: bool = False) -> int:
    """1 if ei_loss_fwd's fused A launch takes the band-sums form (the
    kernels of proj_fwd_multi_ws), 0 for the cluster form (proj_fwd_multi)."""
    mp, mc_m = _idx_rows(plan, mc_idx, B, per_sample)
    sp, sk_m = _idx_rows(plan, sk_idx, B, per_sample)
    rc = int(_lib.skei_ei_fwd_form(plan.handle, B, G, mp, mc_m, sp, sk_m, int(per_sample)))
    _check(rc if rc < 0 else 0, "skei_ei_fwd_form")
    return rc


def _ei_fwd(plan, x1, y, g_deg, mc_idx, sk_idx, work, out, per_sample):
    B, G = x1.shape[0], g_deg.shape[1]
    mp, mc_m = _idx_rows(plan, mc_idx, B, per_sample)
    sp, sk_m = _idx_rows(plan, sk_idx, B, per_sample)
    N, nd = plan.N, plan.n_det
    _dev(x1, "x1", shape=(B, N, N))
    _dev(y, "y", x1.dtype, (B, plan.n_angles, nd))
    _dev(g_deg, "g_deg", torch.float64, (B, G))
    if out is None:
        out = (torch.empty((B, mc_m, nd), device=x1.device, dtype=x1.dtype),
               torch.empty((B, G, N, N), device=x1.device, dtype=x1.dtype),
               torch.empty((B, G, N, N), device=x1.device, dtype=x1.dtype))
    r, x2, z = out
    _dev(r, "r", x1.dtype, (B, mc_m, nd))
    _dev(x2, "x2", x1.dtype, (B, G, N, N))
    _dev(z, "z", x1.dtype, (B, G, N, N))
    code = _dtype_code(x1)
    nb = ei_workspace_size(plan, code, B, G, mc_m, sk_m)
    w = _work(nb, x1.device, work)
    fn = _lib.skei_ei_loss_fwd_per_sample if per_sample else _lib.skei_ei_loss_fwd
    _check(fn(plan.handle, code, _ptr(x1), _ptr(y), B, mp, mc_m, sp, sk_m, _ptr(g_deg), G,
              _ptr(r), _ptr(x2), _ptr(z), _ptr(w), nb, _stream()),
           "skei_ei_loss_fwd_per_sample" if per_sample else "skei_ei_loss_fwd")
    return r, x2, z


def ei_loss_fwd(plan: Plan, x1, y, g_deg, mc_idx=None, sk_idx=None, work=None, out=None):
    """Stage 1 of the (sketched) EI loss.  Returns (r, x2, z)."""
    return _ei_fwd(plan, x1, y, g_deg, mc_idx, sk_idx, work, out, False)


def ei_loss_fwd_per_sample(plan: Plan, x1, y, g_deg, mc_idx=None, sk_idx=None, work=None,
                           out=None):
    """Stage 1 with an angle list per measurement: mc_idx, sk_idx int32 [B, m]."""
    return _ei_fwd(plan, x1, y, g_deg, mc_idx, sk_idx, work, out, True)


def ei_loss_finish(x2, x3, r, lam: float, mc_scale: float, want_grads=True, work=None,
                   out=None):
    """Returns (loss[1], mc[B], ei[B, G], g_x2, g_x3) with FP64 sums on the
    device; x2, x3 [B, G, ...] (any image shape), r [B, ...]."""
    B, G = x2.shape[0], x2.shape[1]
    _dev(x2, "x2")
    _dev(x3, "x3", x2.dtype, x2.shape)
    _dev(r, "r", x2.dtype)
    img_len = x2[0, 0].numel()
    r_len = r.numel() // B
    dev = x2.device
    if out is None:
        out = (torch.empty(1, dtype=torch.float64, device=dev),
               torch.empty(B, dtype=torch.float64, device=dev),
               torch.empty((B, G), dtype=torch.float64, device=dev),
               torch.empty_like(x2) if want_grads else None,
               torch.empty_like(x2) if want_grads else None)
    loss, mc, ei, g_x2, g_x3 = out
    nb = int(_lib.skei_ei_finish_len_workspace_size(B, G, img_len, r_len))
    w = _work(nb, dev, work)
    _check(_lib.skei_ei_loss_finish_len(_dtype_code(x2), _ptr(x2), _ptr(x3), _ptr(r), B, G,
                                        img_len, r_len, float(lam), float(mc_scale), _ptr(mc),
                                        _ptr(ei), _ptr(loss), _ptr(g_x2), _ptr(g_x3), _ptr(w), nb,
                                        _stream()), "skei_ei_loss_finish_len")
    return loss, mc, ei, g_x2, g_x3


def _ei_bwd(plan, r, g_x2, g_z, g_deg, mc_coef, mc_idx, sk_idx, work, out, per_sample):
    B, G = g_deg.shape
    mp, mc_m = _idx_rows(plan, mc_idx, B, per_sample)
    sp, sk_m = _idx_rows(plan, sk_idx, B, per_sample)
    N, nd = plan.N, plan.n_det
    _dev(r, "r", shape=(B, mc_m, nd))
    _dev(g_x2, "g_x2", r.dtype, (B, G, N, N))
    _dev(g_z, "g_z", r.dtype, (B, G, N, N))
    _dev(g_deg, "g_deg", torch.float64, (B, G))
    out = torch.empty((B, N, N), device=r.device, dtype=r.dtype) if out is None else out
    _dev(out, "out", r.dtype, (B, N, N))
    code = _dtype_code(r)
    nb = ei_workspace_size(plan, code, B, G, mc_m, sk_m)
    w = _work(nb, r.device, work)
    fn = _lib.skei_ei_loss_bwd_per_sample if per_sample else _lib.skei_ei_loss_bwd
    _check(fn(plan.handle, code, _ptr(r), _ptr(g_x2), _ptr(g_z), B, mp, mc_m, sp, sk_m,
              _ptr(g_deg), G, float(mc_coef), _ptr(out), _ptr(w), nb, _stream()),
           "skei_ei_loss_bwd_per_sample" if per_sample else "skei_ei_loss_bwd")
    return out


def ei_loss_bwd(plan: Plan, r, g_x2, g_z, g_deg, mc_coef: float, mc_idx=None, sk_idx=None,
                work=None, out=None):
    """g_x1 = -2 mc_coef A_mc^T r + sum_g T_g^T [g_x2 + (pi/m) A_S^T H B_S^T g_z]."""
    return _ei_bwd(plan, r, g_x2, g_z, g_deg, mc_coef, mc_idx, sk_idx, work, out, False)


def ei_loss_bwd_per_sample(plan: Plan, r, g_x2, g_z, g_deg, mc_coef: float, mc_idx=None,
                           sk_idx=None, work=None, out=None):
    """The same with an angle list per measurement: mc_idx, sk_idx int32 [B, m]."""
    return _ei_bwd(plan, r, g_x2, g_z, g_deg, mc_coef, mc_idx, sk_idx, work, out, True)


def residual_add(u, theta, out=None) -> torch.Tensor:
    """u + theta, theta (float32, n elements) broadcast over the leading dims of u."""
    n = theta.numel()
    if u.numel() % n:
        raise ValueError("u.numel() must be a multiple of theta.numel()")
    _dev(u, "u")
    _dev(theta, "theta", torch.float32)
    out = torch.empty_like(u) if out is None else out
    _dev(out, "out", u.dtype, u.shape)
    _check(_lib.skei_residual_add(_dtype_code(u), _ptr(u), _ptr(theta), u.numel() // n, n,
                                  _ptr(out), _stream()), "skei_residual_add")
    return out


def adam_step(theta, m, v, step_dev, g1, g2=None, lr=5e-4, beta1=0.9, beta2=0.999, eps=1e-8):
    """In-place Adam on theta/m/v (float32) with g = sum over leading dims of
    g1 (and g2); step_dev is a CUDA int32 scalar tensor (>= 1)."""
    n = theta.numel()
    for t, nm in ((theta, "theta"), (m, "m"), (v, "v")):
        _dev(t, nm, torch.float32)
    _dev(step_dev, "step", torch.int32)
    _dev(g1, "g1")
    c1 = g1.numel() // n
    c2 = 0 if g2 is None else g2.numel() // n
    if g2 is not None:
        _dev(g2, "g2", g1.dtype)
    _check(_lib.skei_adam_step(_ptr(theta), n, _dtype_code(g1), _ptr(g1), c1, _ptr(g2), c2,
                               _ptr(m), _ptr(v), _ptr(step_dev), lr, beta1, beta2, eps, _stream()),
           "skei_adam_step")


def ttt_residual_workspace_size(plan: Plan, dtype: int, B: int, G: int, mc_m: int,
                                sk_m: int) -> int:
    return int(_lib.skei_ttt_residual_workspace_size(plan.handle, dtype, B, G, mc_m, sk_m))


def ttt_residual_step(plan: Plan, x0, theta, m, v, step_dev, y, g_deg, mc_idx=None, sk_idx=None,
                      lam=1.0, mc_scale=1.0, lr=5e-4, beta1=0.9, beta2=0.999, eps=1e-8,
                      out=None, work=None):
    """skei_ttt_residual_step: Algorithm 2's iteration for F(u) = u + theta
    (theta, m, v updated in place).  out = (x1, r, x2, z, x3, g_x2, g_x3, g_x1,
    loss, mc, ei), allocated when None; returns it."""
    B, G = x0.shape[0], g_deg.shape[1]
    mp, mc_m = _idx_rows(plan, mc_idx, B, False)
    sp, sk_m = _idx_rows(plan, sk_idx, B, False)
    N, nd = plan.N, plan.n_det
    _dev(x0, "x0", shape=(B, N, N))
    _dev(y, "y", x0.dtype, (B, plan.n_angles, nd))
    _dev(g_deg, "g_deg", torch.float64, (B, G))
    for t, nm in ((theta, "theta"), (m, "m"), (v, "v")):
        _dev(t, nm, torch.float32, (N, N))
    _dev(step_dev, "step", torch.int32)
    dev, dt = x0.device, x0.dtype
    if out is None:
        img = lambda *sh: torch.empty(sh, device=dev, dtype=dt)  # noqa: E731
        out = (img(B, N, N), img(B, mc_m, nd), img(B, G, N, N), img(B, G, N, N),
               img(B, G, N, N), img(B, G, N, N), img(B, G, N, N), img(B, N, N),
               torch.empty(1, device=dev, dtype=torch.float64),
               torch.empty(B, device=dev, dtype=torch.float64),
               torch.empty((B, G), device=dev, dtype=torch.float64))
    x1, r, x2, z, x3, gx2, gx3, gx1, loss, mc, ei = out
    for t, nm, sh in ((x1, "x1", (B, N, N)), (r, "r", (B, mc_m, nd)), (x2, "x2", (B, G, N, N)),
                      (z, "z", (B, G, N, N)), (x3, "x3", (B, G, N, N)),
                      (gx2, "g_x2", (B, G, N, N)), (gx3, "g_x3", (B, G, N, N)),
                      (gx1, "g_x1", (B, N, N))):
        _dev(t, nm, dt, sh)
    code = _dtype_code(x0)
    nb = ttt_residual_workspace_size(plan, code, B, G, mc_m, sk_m)
    w = _work(nb, dev, work)
    _check(_lib.skei_ttt_residual_step(
        plan.handle, code, _ptr(x0), _ptr(theta), _ptr(m), _ptr(v), _ptr(step_dev), _ptr(y), B,
        mp, mc_m, sp, sk_m, _ptr(g_deg), G, float(lam), float(mc_scale), float(lr), float(beta1),
        float(beta2), float(eps), _ptr(x1), _ptr(r), _ptr(x2), _ptr(z), _ptr(x3), _ptr(gx2),
        _ptr(gx3), _ptr(gx1), _ptr(mc), _ptr(ei), _ptr(loss), _ptr(w), nb, _stream()),
        "skei_ttt_residual_step")
    return out


def step_draws(table, counter, out):
    """On the device: out = row counter of table [n_rows, ...] (bytes of one
    row), then counter += 1; a counter outside [0, n_rows) copies nothing and
    becomes -1.  counter is a CUDA int32 tensor of one element."""
    _dev(table, "table")
    _dev(counter, "counter", torch.int32, (1,))
    _dev(out, "out")
    if table.dim() < 2:
        raise ValueError("table must be [n_rows, ...]")
    row_bytes = table[0].numel() * table.element_size()
    if out.numel() * out.element_size() != row_bytes:
        raise ValueError(f"out holds {out.numel() * out.element_size()} bytes, a row {row_bytes}")
    _check(_lib.skei_step_draws(_ptr(table), table.shape[0], row_bytes, _ptr(counter), _ptr(out),
                                _stream()), "skei_step_draws")


# ------------------------------------------------------ batch-norm layers
def _bn_shape(v):
    if v.dim() < 2:
        raise ValueError("v must be [B, C, ...]")
    B, C = v.shape[0], v.shape[1]
    return B, C, v[0, 0].numel()


def bn_workspace_size(B: int, C: int, HW: int) -> int:
    return int(_lib.skei_bn_workspace_size(B, C, HW))


def bn_act_fwd(v, scale, shift, relu=True, eps=1e-5, out=None, work=None):
    """Batch-statistics BN of v [B, C, ...] per channel, then scale/shift
    (float32 [C]) and ReLU (relu=True): returns (out, mean, rstd)."""
    _dev(v, "v")
    B, C, HW = _bn_shape(v)
    _dev(scale, "scale", torch.float32, (C,))
    _dev(shift, "shift", torch.float32, (C,))
    out = torch.empty_like(v) if out is None else out
    _dev(out, "out", v.dtype, v.shape)
    mean = torch.empty(C, dtype=torch.float32, device=v.device)
    rstd = torch.empty_like(mean)
    nb = bn_workspace_size(B, C, HW)
    w = _work(nb, v.device, work)
    _check(_lib.skei_bn_act_fwd(_dtype_code(v), _ptr(v), B, C, HW, _ptr(scale), _ptr(shift),
                                int(bool(relu)), float(eps), _ptr(out), _ptr(mean), _ptr(rstd),
                                _ptr(w), nb, _stream()), "skei_bn_act_fwd")
    return out, mean, rstd


def bn_act_bwd(v, g_out, scale, shift, mean, rstd, relu=True, work=None):
    """Gradients of bn_act_fwd: returns (g_v, g_scale, g_shift)."""
    _dev(v, "v")
    B, C, HW = _bn_shape(v)
    _dev(g_out, "g_out", v.dtype, v.shape)
    for t, nm in ((scale, "scale"), (shift, "shift"), (mean, "mean"), (rstd, "rstd")):
        _dev(t, nm, torch.float32, (C,))
    g_v = torch.empty_like(v)
    g_scale = torch.empty(C, dtype=torch.float32, device=v.device)
    g_shift = torch.empty_like(g_scale)
    nb = bn_workspace_size(B, C, HW)
    w = _work(nb, v.device, work)
    _check(_lib.skei_bn_act_bwd(_dtype_code(v), _ptr(v), _ptr(g_out), B, C, HW, _ptr(scale),
                                _ptr(shift), _ptr(mean), _ptr(rstd), int(bool(relu)), _ptr(g_v),
                                _ptr(g_scale), _ptr(g_shift), _ptr(w), nb, _stream()),
           "skei_bn_act_bwd")
    return g_v, g_scale, g_shift


# --------------------------------------------------------- multi-coil MRI
def mri_workspace_size(N: int, Nc: int, B: int) -> int:
    return int(_lib.skei_mri_workspace_size(N, Nc, B))


def _mri_dims(maps):
    _dev(maps, "maps", torch.float32)
    if maps.dim() != 4 or maps.shape[1] != 2 or maps.shape[2] != maps.shape[3]:
        raise ValueError("maps must be [Nc, 2, N, N]")
    return maps.shape[0], maps.shape[-1]


def mri_fwd(x, maps, mask=None, aux=None, alpha=1.0, xw=None, out=None, work=None):
    """k = alpha (aux - M F (C (xw x))) or alpha M F (C (xw x)); x [B, 2, N, N]
    planar, xw a real [N, N] weight (None = 1)."""
    Nc, N = _mri_dims(maps)
    B = x.shape[0]
    _dev(x, "x", torch.float32, (B, 2, N, N))
    if mask is not None:
        _dev(mask, "mask", torch.float32, (N, N))
    if aux is not None:
        _dev(aux, "aux", torch.float32, (B, Nc, 2, N, N))
    if xw is not None:
        _dev(xw, "xw", torch.float32, (N, N))
    out = torch.empty((B, Nc, 2, N, N), dtype=torch.float32, device=x.device) \
        if out is None else out
    _dev(out, "out", torch.float32, (B, Nc, 2, N, N))
    nb = mri_workspace_size(N, Nc, B)
    w = _work(nb, x.device, work)
    _check(_lib.skei_mri_fwd(N, Nc, B, _ptr(x), _ptr(maps), _ptr(mask), _ptr(xw), _ptr(aux),
                             float(alpha), _ptr(out), _ptr(w), nb, _stream()), "skei_mri_fwd")
    return out


def mri_adj(k, maps, mask=None, dinv=None, alpha=1.0, beta=0.0, out=None, work=None):
    """x = alpha dinv sum_c conj(C_c) F^H (M k_c) + beta x; k [B, Nc, 2, N, N]."""
    Nc, N = _mri_dims(maps)
    B = k.shape[0]
    _dev(k, "k", torch.float32, (B, Nc, 2, N, N))
    if mask is not None:
        _dev(mask, "mask", torch.float32, (N, N))
    if dinv is not None:
        _dev(dinv, "dinv", torch.float32, (N, N))
    out = torch.empty((B, 2, N, N), dtype=torch.float32, device=k.device) if out is None else out
    _dev(out, "out", torch.float32, (B, 2, N, N))
    nb = mri_workspace_size(N, Nc, B)
    w = _work(nb, k.device, work)
    _check(_lib.skei_mri_adj(N, Nc, B, _ptr(k), _ptr(maps), _ptr(mask), _ptr(dinv), float(alpha),
                             float(beta), _ptr(out), _ptr(w), nb, _stream()), "skei_mri_adj")
    return out


def mri_dinv(maps, out=None):
    Nc, N = _mri_dims(maps)
    out = torch.empty((N, N), dtype=torch.float32, device=maps.device) if out is None else out
    _dev(out, "out", torch.float32, (N, N))
    _check(_lib.skei_mri_dinv(N, Nc, _ptr(maps), _ptr(out), _stream()), "skei_mri_dinv")
    return out


def coil_mix(W, x, out=None):
    """out[b, j] = sum_i W[j, i] x[b, i] for complex W (complex64 [n_out, n_in]
    or float32 [n_out, n_in, 2]) and planar coil data x [B, n_in, 2, ...]."""
    if W.is_complex():
        W = torch.view_as_real(W.to(torch.complex64)).contiguous()
    _dev(W, "W", torch.float32)
    n_out, n_in = W.shape[0], W.shape[1]
    _dev(x, "x", torch.float32)
    if x.dim() < 3 or x.shape[1] != n_in or x.shape[2] != 2:
        raise ValueError("x must be [B, n_in, 2, ...]")
    B, plane = x.shape[0], x[0, 0, 0].numel()
    shape = (B, n_out, 2) + tuple(x.shape[3:])
    out = torch.empty(shape, dtype=torch.float32, device=x.device) if out is None else out
    _dev(out, "out", torch.float32, shape)
    _check(_lib.skei_coil_mix(plane, B, n_in, n_out, _ptr(W), _ptr(x), _ptr(out), _stream()),
           "skei_coil_mix")
    return out


# ------------------------------------------------------- batched schedule
PROJ_FWD, PROJ_ADJ, BACKPROJECT, BACKPROJECT_ADJ, FILTER, FBP = range(6)
_BATCH_NAMES = ["proj_fwd", "proj_adj", "backproject", "backproject_adj", "filter", "fbp"]


class BatchItem:
    """One instance of a batch: `inp` -> `out` under the batch's operator with
    the plan's geometry and the sketch `idx` (int32 CUDA tensor, None = all
    angles); out = scale * op(inp)."""

    def __init__(self, plan: Plan, inp, out, idx=None, scale: float = 1.0):
        self.plan, self.inp, self.out, self.idx, self.scale = plan, inp, out, idx, float(scale)


class Batch:
    """skei_batch_*: one operator over many instances (different plans,
    sketches and storage types) in one persistent launch per kernel.  The
    tensors are baked in at creation: write new inputs into them and call
    run() again (also inside a captured CUDA graph)."""

    def __init__(self, op: int, items):
        if op not in range(6):
            raise ValueError(f"unknown batch operator {op}")
        self.op, self.items = op, list(items)
        arr = (_BatchItemC * len(self.items))()
        for q, it in enumerate(self.items):
            p = it.plan
            idx_p, m = _idx(p, it.idx)
            B = int(it.inp.shape[0]) if it.inp.dim() >= 1 else 0
            img, sino = (B, p.N, p.N), (B, m, p.n_det)
            shp_in, shp_out = {
                PROJ_FWD: (img, sino), PROJ_ADJ: (sino, img), BACKPROJECT: (sino, img),
                BACKPROJECT_ADJ: (img, sino), FILTER: (sino, sino), FBP: (sino, img)}[op]
            _dev(it.inp, f"items[{q}].inp", shape=shp_in)
            _dev(it.out, f"items[{q}].out", shape=shp_out)
            arr[q] = _BatchItemC(p.handle.value, _dtype_code(it.inp), _dtype_code(it.out),
                                 it.inp.data_ptr(), it.out.data_ptr(),
                                 None if idx_p is None else idx_p.value, m, B, it.scale)
        self._h = _BATCH()
        _check(_lib.skei_batch_create(int(op), arr, len(self.items), ctypes.byref(self._h)),
               "skei_batch_create")

    @property
    def handle(self):
        if not self._h:
            raise RuntimeError("batch is closed")
        return self._h

    def run(self) -> None:
        _check(_lib.skei_batch_run(self.handle, _stream()), "skei_batch_run")

    def tune(self, reps: int = 5) -> None:
        _check(_lib.skei_batch_tune(self.handle, int(reps), _stream()), "skei_batch_tune")

    def info(self, phase: int = 0) -> dict:
        n_ph, n_t, w, blk = _i(), _i(), _i(), _i()
        _check(_lib.skei_batch_info(self.handle, int(phase), ctypes.byref(n_ph), ctypes.byref(n_t),
                                    ctypes.byref(w), ctypes.byref(blk)), "skei_batch_info")
        return {"phases": n_ph.value, "tasks": n_t.value, "workers": w.value, "block": blk.value}

    def close(self):
        if self._h:
            _lib.skei_batch_destroy(self._h)
            self._h = _BATCH()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def measure_roofs(work=None) -> dict:
    """skei_measure_roofs: measured FP32 FMA rate (flop/s), shared-memory load
    bandwidth, L2 and DRAM read bandwidths (bytes/s) on the current device and
    stream.  `work` is a CUDA byte tensor of >= ROOFS_WORK_BYTES (allocated
    here when omitted).  Synchronises the stream."""
    work = _work(ROOFS_WORK_BYTES, torch.device("cuda", torch.cuda.current_device()), work)
    out = _Roofs()
    _check(_lib.skei_measure_roofs(_ptr(work), work.numel(), ctypes.byref(out), _stream()),
           "skei_measure_roofs")
    return {"fp32_flops": out.fp32_flops, "smem_bytes": out.smem_bytes,
            "l2_bytes": out.l2_bytes, "dram_read_bytes": out.dram_read_bytes, "sms": out.sms}


def check_build() -> bool:
    """Whether the loaded library is the bounds-check build."""
    return bool(_lib.skei_check_build())


def check_status(reset: bool = True) -> int:
    """skei_check_status: the range-check bits seen since the last reset (0
    in the normal build); synchronises the device."""
    bits = ctypes.c_uint(0)
    _check(_lib.skei_check_status(ctypes.byref(bits), int(reset)), "skei_check_status")
    return bits.value
