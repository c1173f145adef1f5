"""Small cases of every instrumented kernel family, run against the
bounds-check build of the library (libskei_check.so, SKEI_CHECK = 1; the
caller sets SKEI_LIBRARY): the cluster and band-sums forms of A and B^T (a
riding image, groups of 4 and single images, ragged N), the tile kernels
(A^T, B), the filter (direct, fused with the band sums in the step) and the
one-call TTT step.  Every output sits between NaN guard bands that no
kernel may touch; every result is compared with the FP64 oracle; at the end
the device check word must be zero.  Prints CHECK_OK on success."""
import os
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle as O  # noqa: E402
from paper_2411_05771_gb300 import inputs as I  # noqa: E402
from paper_2411_05771_gb300 import skei as S  # noqa: E402

GUARD = 1024
TOL = 1e-5
_guards = []


def guarded(shape, dtype=torch.float32):
    """A CUDA tensor of `shape` inside a buffer with GUARD NaN elements on
    each side (checked at the end)."""
    n = int(np.prod(shape))
    buf = torch.full((n + 2 * GUARD,), float("nan"), dtype=dtype, device="cuda")
    _guards.append(buf)
    return buf[GUARD:GUARD + n].view(shape)


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def host(t):
    return t.detach().double().cpu().numpy()


def dev(a, dtype=torch.float32):
    return torch.tensor(np.asarray(a), dtype=dtype, device="cuda")


def check(name, got, ref, tol=TOL):
    e = rel(host(got), ref)
    assert e <= tol, f"{name}: rel-L2 {e:.3g} > {tol}"


def operators(N, n_ang, B, m, seed):
    rng = np.random.default_rng(seed)
    plan = S.Plan(N, n_ang)
    nd = plan.n_det
    idx_np = I.sketch_indices(n_ang, m, int(rng.integers(0, n_ang // m))) if m < n_ang else None
    idx = None if idx_np is None else dev(idx_np, torch.int32)
    ang = plan.angles_deg if idx_np is None else O.select(plan.angles_deg, idx_np)
    x = rng.standard_normal((B, N, N))
    p = rng.standard_normal((B, m, nd))
    xd, pd = dev(x), dev(p)
    # A: cluster form; band sums with a riding image (B images, 4 B images)
    check("A", S.proj_fwd(plan, xd, idx, out=guarded((B, m, nd))), O.proj_fwd(x, ang, nd))
    x4 = rng.standard_normal((4 * B, N, N))
    jobs = [S.Job(xd, guarded((B, m, nd)), idx), S.Job(dev(x4), guarded((4 * B, m, nd)), idx)]
    S.proj_fwd_multi_ws(plan, jobs)
    check("A riding", jobs[0].out, O.proj_fwd(x, ang, nd))
    check("A group", jobs[1].out, O.proj_fwd(x4, ang, nd))
    # A^T, B, B^T (cluster and band sums), H, FBP
    check("A^T", S.proj_adj(plan, pd, idx, out=guarded((B, N, N))), O.proj_adj(p, ang, N))
    check("B", S.backproject(plan, pd, idx, out=guarded((B, N, N))), O.backproject(p, ang, N))
    check("B^T", S.backproject_adj(plan, xd, idx, out=guarded((B, m, nd))),
          O.backproject_adj(x, ang, nd))
    jb = [S.Job(dev(x4), guarded((4 * B, m, nd)), idx)]
    S.backproject_adj_multi_ws(plan, jb)
    check("B^T group", jb[0].out, O.backproject_adj(x4, ang, nd))
    check("H", S.filter(plan, pd, 0.5, out=guarded((B, m, nd))), 0.5 * O.ramlak(p))
    check("FBP", S.fbp(plan, pd, idx, out=guarded((B, N, N))), O.fbp(p, ang, N))


def ttt_step(N, n_ang, G, m, seed):
    rng = np.random.default_rng(seed)
    plan = S.Plan(N, n_ang)
    nd = plan.n_det
    idx_np = I.sketch_indices(n_ang, m, int(rng.integers(0, n_ang // m)))
    idx = dev(idx_np, torch.int32)
    x0 = I.rasterize(I.random_ellipses(seed), N)[None]
    y = rng.standard_normal((1, n_ang, nd))
    g = I.rotation_angles(rng, 1, G)
    theta = 0.01 * rng.standard_normal((N, N))
    th = dev(theta)
    mm, vv = torch.zeros_like(th), torch.zeros_like(th)
    step = torch.ones((), dtype=torch.int32, device="cuda")
    out = (guarded((1, N, N)), guarded((1, m, nd)), guarded((1, G, N, N)), guarded((1, G, N, N)),
           guarded((1, G, N, N)), guarded((1, G, N, N)), guarded((1, G, N, N)),
           guarded((1, N, N)), guarded((1,), torch.float64), guarded((1,), torch.float64),
           guarded((1, G), torch.float64))
    S.ttt_residual_step(plan, dev(x0), th, mm, vv, step, dev(y), dev(g, torch.float64), idx, idx,
                        1.0, n_ang / m, out=out)
    x1 = x0 + theta[None]
    r, x2, z = O.ei_stage1(x1, y, plan.angles_deg, idx_np, idx_np, g)
    x3 = z + theta[None, None]
    loss, mc, ei, gx2, gx3 = O.ei_finish(x2, x3, r, 1.0, n_ang / m)
    gx1 = O.ei_backward(r, gx2, gx3, plan.angles_deg, idx_np, idx_np, g, n_ang / m)
    y_mc = y[:, idx_np]
    assert np.linalg.norm(host(out[1]) - r) <= TOL * np.linalg.norm(y_mc), "step: r"
    for name, got, ref in (("x2", out[2], x2), ("z", out[3], z), ("x3", out[4], x3),
                           ("g_x2", out[5], gx2), ("g_x1", out[7], gx1), ("ei", out[10], ei)):
        check("step " + name, got, ref)
    assert abs(out[8].item() - loss) <= TOL * abs(loss), "step: loss"


def main():
    assert S.check_build(), "SKEI_LIBRARY does not name the bounds-check build"
    S.check_status(reset=True)
    for case in ((37, 24, 3, 8, 1), (64, 60, 5, 15, 2), (8, 12, 1, 12, 3), (100, 30, 2, 10, 4)):
        operators(*case)
    ttt_step(64, 60, 4, 15, 5)
    ttt_step(37, 24, 3, 6, 6)
    torch.cuda.synchronize()
    bits = S.check_status()
    assert bits == 0, f"out-of-range accesses: check word {bits:#x}"
    for buf in _guards:
        assert bool(torch.isnan(buf[:GUARD]).all()) and bool(torch.isnan(buf[-GUARD:]).all()), \
            "a kernel wrote into a NaN guard band"
    print("CHECK_OK")


if __name__ == "__main__":
    main()
