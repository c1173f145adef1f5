"""Benchmark: sketched-EI test-time-training steps/s at 512^2 on GB300.

Workload (the TTT-shaped run of the paper's CT experiments, synthetic): a
512x512 phantom of 10 random ellipses; a 60-view parallel-beam sinogram with
725 bins from the analytic Radon transform, Poisson noise at I0 = 1e5 plus
Gaussian sigma = 0.01 (post-log); x0 = FBP(y); stand-in network
F(u) = u + theta; per step one interleaved 30-angle sketch (random offset)
and G = 4 rotations U[0, 360); loss Eq. (e:skeilossttt) forward + hand-
written backward + Adam (lr 5e-4) - Algorithm 2's iteration.

The sketched arm (the headline value) is compared with the plain full-
operator EI step (all 60 angles) on the same GPU, and both are run for 200
iterations from the same start to compare reconstruction PSNR.

Contract: `python bench.py --gpus N --steps K --warmup W` prints one JSON
line; N>1 runs under torchrun, one independent replica per GPU (weak
scaling).  `--impl reference` times the FP64 CPU oracle on the same step.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "EI-loss steps/s, sketched vs plain, 512² at equal PSNR; A/Aᵀ % of roofline"
UNIT = "steps/s"

# workload
N_IMG, N_VIEWS, SKETCH, G_ROT, BATCH = 512, 60, 30, 4, 1
LAM, LR = 1.0, 5e-4
PSNR_ITERS = 1000          # iterations of each arm's PSNR trajectory
PSNR_REF_ITERS = 200       # the TTT run length of the equal-PSNR comparison
L2_FLUSH_BYTES = 256 << 20
MIN_TIMED_S = 1.0          # device time the timed region lasts at the least
MAX_TIMED_STEPS = 20000


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="skei", choices=["skei", "reference"])
    ap.add_argument("--dtype", default="f32", choices=["f32", "bf16"],
                    help="storage type of the sketched arm")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-steps", type=int, default=0, help="oracle steps (0 = auto, ~15 s)")
    ap.add_argument("--suite", action="store_true",
                    help="instead of the headline line, print one JSON line per measurement "
                         "of the other workloads: single operators at 64^2 and 8 x 256^2, the "
                         "differentiated EI step at 8 x 4 x 256^2, the 16-instance batch")
    ap.add_argument("--profile", action="store_true",
                    help="set up the sketched arm, run one warm and one more step, then each "
                         "operator of the kernel breakdown once, and exit (a short, untimed run "
                         "for ncu; it prints its launch counts)")
    return ap.parse_args()


# --------------------------------------------------------------------- inputs
class Workload:
    """Shape of one TTT step: B images of N^2, `views` angles, EI term on an
    m-angle interleaved sketch (m = views: no sketch), MC term on the same
    sketch or on all views, G rotations per image."""

    def __init__(self, N=N_IMG, views=N_VIEWS, m=SKETCH, G=G_ROT, B=BATCH, mc_sketched=True,
                 noisy=True, draw_m=None, per_sample=False):
        self.N, self.views, self.m, self.G, self.B = N, views, m, G, B
        # per_sample: every measurement draws its own sketch (Algorithm 1)
        self.per_sample = per_sample and m < views
        self.mc_sketched = mc_sketched and m < views
        self.noisy = noisy
        # sketch size of the per-step offset draw: the plain arm draws as the
        # sketched one does, so both see the same rotations
        self.draw_m = draw_m or m

    @property
    def sketched(self):
        return self.m < self.views

    @property
    def mc_m(self):
        return self.m if self.mc_sketched else self.views

    @property
    def mc_scale(self):
        return self.views / self.m if self.mc_sketched else 1.0


SKETCHED = Workload()                                   # the headline arm
PLAIN = Workload(m=N_VIEWS, mc_sketched=False, draw_m=SKETCH)   # full operators


def workload_config():
    """The workload keys both arms of the bench report."""
    n_det = int(np.ceil(N_IMG * np.sqrt(2.0))) | 1
    return {"workload": f"ttt-{N_IMG}x{N_IMG}-{N_VIEWS}views-{n_det}bins-sketch{SKETCH}-G{G_ROT}",
            "N": N_IMG, "views": N_VIEWS, "n_det": n_det, "sketch": SKETCH, "G": G_ROT,
            "B": BATCH, "lambda": LAM, "network": "F(u)=u+theta", "optimizer": "adam lr 5e-4"}


def make_problem(wl=SKETCHED, seed=0):
    from paper_2411_05771_gb300 import inputs as I
    angs = I.uniform_angles(wl.views)
    n_det = int(np.ceil(wl.N * np.sqrt(2.0))) | 1
    xs, ys = [], []
    for b in range(wl.B):
        e = I.random_ellipses(seed + b)
        xs.append(I.rasterize(e, wl.N))
        y = I.analytic_sinogram(e, wl.N, angs, n_det)
        ys.append(I.noisy_sinogram(y, wl.N, seed=seed + b + 77) if wl.noisy else y)
    return dict(x_gt=xs[0], x_all=np.stack(xs), angs=angs, n_det=n_det, y=ys[0], y_all=np.stack(ys))


def step_params(n_steps, wl, first=0):
    """Per-step draws (Algorithm 2): one sketch offset (one per measurement
    with per_sample, Algorithm 1) and B x G rotation angles from
    default_rng(1000 + step)."""
    from paper_2411_05771_gb300 import inputs as I
    idx, g = [], []
    for s in range(first, first + n_steps):
        rng = I.step_rng(s)
        if wl.per_sample:
            idx.append(np.stack([I.sketch_indices(wl.views, wl.m,
                                                  I.random_sketch_offset(rng, wl.views, wl.draw_m))
                                 for _ in range(wl.B)]))
        else:
            off = I.random_sketch_offset(rng, wl.views, wl.draw_m)
            idx.append(I.sketch_indices(wl.views, wl.m, off) if wl.sketched
                       else np.arange(wl.views, dtype=np.int32))
        g.append(I.rotation_angles(rng, wl.B, wl.G))
    return np.stack(idx).astype(np.int32), np.stack(g)


# ------------------------------------------------------------------ GPU arm
class Arm:
    """One TTT problem on the GPU with all buffers resident; `step()` issues
    Algorithm 2's iteration through the C ABI on the current stream."""

    def __init__(self, S, plan, prob, wl, dtype, device):
        import torch
        self.S, self.plan, self.wl = S, plan, wl
        self.sketched = wl.sketched
        self.tdt = torch.float32 if dtype == "f32" else torch.bfloat16
        N, nd, B, G = wl.N, plan.n_det, wl.B, wl.G
        self.m, self.mc_m = wl.m, wl.mc_m
        self.mc_scale = wl.mc_scale
        d = device
        self.y = torch.tensor(prob["y_all"], dtype=self.tdt, device=d)
        y32 = torch.tensor(prob["y_all"], dtype=torch.float32, device=d)
        self.x0 = S.fbp(plan, y32).to(self.tdt).contiguous()
        self.theta = torch.zeros((N, N), dtype=torch.float32, device=d)
        self.m1 = torch.zeros_like(self.theta)
        self.v1 = torch.zeros_like(self.theta)
        # the step's draws live in one device buffer (rotation angles, sketch
        # rows, step number), so that a step uploads them with one copy
        self.g_off, self.idx_off = 0, 8 * B * G
        self.step_off = self.idx_off + 4 * self.m * (B if wl.per_sample else 1)
        self.param_bytes = (self.step_off + 4 + 15) // 16 * 16
        self.params = torch.zeros(self.param_bytes, dtype=torch.uint8, device=d)
        self.g = self.params[self.g_off:self.idx_off].view(torch.float64).view(B, G)
        self.idx = self.params[self.idx_off:self.step_off].view(torch.int32)
        if wl.per_sample:
            self.idx = self.idx.view(B, self.m)
        self.step_no = self.params[self.step_off:self.step_off + 4].view(torch.int32)
        self.x1 = torch.empty((B, N, N), dtype=self.tdt, device=d)
        self.r = torch.empty((B, self.mc_m, nd), dtype=self.tdt, device=d)
        self.x2 = torch.empty((B, G, N, N), dtype=self.tdt, device=d)
        self.z = torch.empty_like(self.x2)
        self.x3 = torch.empty_like(self.x2)
        self.gx2 = torch.empty_like(self.x2)
        self.gx3 = torch.empty_like(self.x2)
        self.gx1 = torch.empty_like(self.x1)
        self.loss = torch.empty(1, dtype=torch.float64, device=d)
        self.mc = torch.empty(B, dtype=torch.float64, device=d)
        self.ei = torch.empty((B, G), dtype=torch.float64, device=d)
        code = S.F32 if dtype == "f32" else S.BF16
        self.work = torch.empty(max(S.ttt_residual_workspace_size(plan, code, B, G, self.mc_m,
                                                                  self.m),
                                    S.ei_workspace_size(plan, code, B, G, self.mc_m, self.m),
                                    16), dtype=torch.uint8, device=d)
        idx_all, g_all = step_params(1, wl)
        self.load_params(idx_all[0], g_all[0], 1)
        # kernels per step (skei_ttt_residual_step): rotation (+ x1) 1, A 2
        # (band sums or clusters, then their reduction with the filter), B
        # (+ x3) 1, loss partials 1, B^T 2, A^T 1, rotation transpose (+ Adam
        # + the loss's final pass) 1; with several measurements the Adam
        # update and the final pass take a launch each
        self.launches_per_step = (9 if B == 1 else 11) if not wl.per_sample else 13

    def pack_params(self, idx_all, g_all, first_step):
        """Host bytes of the draws of consecutive steps, one row per step, in
        the layout of self.params."""
        n = len(idx_all)
        host = np.zeros((n, self.param_bytes), dtype=np.uint8)
        host[:, self.g_off:self.idx_off] = np.ascontiguousarray(
            g_all, dtype=np.float64).reshape(n, -1).view(np.uint8)
        host[:, self.idx_off:self.step_off] = np.ascontiguousarray(
            idx_all, dtype=np.int32).reshape(n, -1).view(np.uint8)
        host[:, self.step_off:self.step_off + 4] = np.arange(
            first_step, first_step + n, dtype=np.int32).reshape(n, 1).view(np.uint8)
        return host

    def load_params(self, idx, g, step_no):
        import torch
        self.idx.copy_(torch.as_tensor(idx))
        self.g.copy_(torch.as_tensor(g))
        self.step_no.fill_(step_no)

    def step(self):
        """Algorithm 2's iteration: x1 = F(x0), the loss forward, its
        backward and Adam on theta (dL/dtheta = dL/dx1 + sum_g dL/dx3, F's
        Jacobian being the identity), in one library call; with a sketch
        per measurement, the separate calls."""
        S, p = self.S, self.plan
        mc_idx = self.idx if self.wl.mc_sketched else None
        sk_idx = self.idx if self.sketched else None
        if not self.wl.per_sample:
            S.ttt_residual_step(p, self.x0, self.theta, self.m1, self.v1, self.step_no, self.y,
                                self.g, mc_idx, sk_idx, LAM, self.mc_scale, LR,
                                out=(self.x1, self.r, self.x2, self.z, self.x3, self.gx2,
                                     self.gx3, self.gx1, self.loss, self.mc, self.ei),
                                work=self.work)
            return
        S.residual_add(self.x0, self.theta, out=self.x1)                      # x1 = F(x0)
        S.ei_loss_fwd_per_sample(p, self.x1, self.y, self.g, mc_idx, sk_idx, work=self.work,
                                 out=(self.r, self.x2, self.z))
        S.residual_add(self.z, self.theta, out=self.x3)                       # x3 = F(z)
        S.ei_loss_finish(self.x2, self.x3, self.r, LAM, self.mc_scale, work=self.work,
                         out=(self.loss, self.mc, self.ei, self.gx2, self.gx3))
        S.ei_loss_bwd_per_sample(p, self.r, self.gx2, self.gx3, self.g,
                                 self.mc_scale / self.wl.B, mc_idx, sk_idx, work=self.work,
                                 out=self.gx1)
        S.adam_step(self.theta, self.m1, self.v1, self.step_no, self.gx1, self.gx3, lr=LR)

    def reset(self):
        self.theta.zero_()
        self.m1.zero_()
        self.v1.zero_()


def psnr_curve(arm, x_gt, iters):
    """Algorithm 2 for `iters` iterations from theta = 0; PSNR of F(x0) =
    x0 + theta against the phantom after every iteration (untimed; the
    squared errors are summed on the device and read back once)."""
    import torch
    arm.reset()
    idx_all, g_all = step_params(iters, arm.wl)
    gt = torch.tensor(x_gt, dtype=torch.float64, device=arm.theta.device)
    sse = torch.empty(iters + 1, dtype=torch.float64, device=gt.device)
    for s in range(iters + 1):
        sse[s] = ((arm.x0[0].double() + arm.theta.double() - gt) ** 2).sum()
        if s == iters:
            break
        arm.load_params(idx_all[s], g_all[s], s + 1)
        arm.step()
    rngv = float(x_gt.max() - x_gt.min())
    mse = sse.cpu().numpy() / x_gt.size
    return {s: float(10 * np.log10(rngv * rngv / mse[s])) for s in range(iters + 1)}


def psnr_block(c_sk, c_pl, ms_sk, ms_pl):
    """Equal-PSNR comparison on trajectories observed after every iteration:
    the first sketched iteration within 0.1 dB of (and the first at or
    above) the plain arm's PSNR after PSNR_REF_ITERS iterations, and of its
    best PSNR over the run; each with the time ratio plain / sketched."""
    ref = c_pl[PSNR_REF_ITERS]
    best_it = max(c_pl, key=c_pl.get)
    best = c_pl[best_it]
    out = {"iters_run": PSNR_ITERS, "sampled": "every iteration", "fbp_x0": c_pl[0],
           "at_ref_iters": {"iters": PSNR_REF_ITERS, "plain": ref, "sketched": c_sk[PSNR_REF_ITERS],
                            "delta_db": c_sk[PSNR_REF_ITERS] - ref},
           "plain_best": {"psnr": best, "iters": best_it},
           "sketched_best": {"psnr": max(c_sk.values()), "iters": max(c_sk, key=c_sk.get)}}
    for key, target, it_pl in (("to_plain_ref", ref, PSNR_REF_ITERS), ("to_plain_best", best, best_it)):
        blk = {"target_db": target, "plain_iters": it_pl, "plain_ms": it_pl * ms_pl}
        for tag, thr in (("within_0.1db", target - 0.1), ("reached", target)):
            it_sk = first_at(c_sk, thr)
            if it_sk is None:
                blk[tag] = None
                continue
            blk[tag] = {"sketched_iters": it_sk, "sketched_psnr": c_sk[it_sk],
                        "delta_db": c_sk[it_sk] - target, "sketched_ms": it_sk * ms_sk,
                        "speedup": (it_pl * ms_pl) / max(it_sk * ms_sk, 1e-30)}
        out[key] = blk
    out["curve_every_100"] = {"plain": {k: round(v, 3) for k, v in c_pl.items() if k % 100 == 0},
                              "sketched": {k: round(v, 3) for k, v in c_sk.items() if k % 100 == 0}}
    return out


def first_at(curve, target):
    """First observed iteration at which the curve is >= target, or None."""
    for it in sorted(curve):
        if curve[it] >= target:
            return it
    return None


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, gpu_id):
        self.path = tempfile.mktemp(suffix=".csv")
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(["nvidia-smi", f"--id={gpu_id}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "50"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
            return
        # start timing only once samples flow (nvidia-smi takes a moment)
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < 5.0 and self.p.poll() is None:
            if os.path.getsize(self.path) > 0:
                break
            time.sleep(0.01)
        self.f.flush()
        self.skip = sum(1 for _ in open(self.path))   # samples taken before the timed region

    def stop(self):
        if not self.p:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for n, line in enumerate(open(self.path)):
            if n < getattr(self, "skip", 0):
                continue
            parts = [t.strip() for t in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def breakdown_ops(S, arm):
    """Every operator of one step as a call through its public entry point
    with the step's own arguments (A and B^T in the band-sums form: sums,
    then their reduction, two launches; the step itself fuses that
    reduction with the filter, and the network and Adam into the rotations
    and the back-projection), by the names the bench reports."""
    import torch
    p = arm.plan
    mc_idx = arm.idx if arm.wl.mc_sketched else None
    sk_idx = arm.idx if arm.sketched else None
    wl = arm.wl
    N, BG, m = wl.N, wl.B * wl.G, arm.m
    f32 = dict(dtype=torch.float32, device="cuda")
    pbuf = torch.empty((BG, m, p.n_det), **f32)
    qbuf = torch.empty_like(pbuf)
    gtot = torch.empty((wl.B, wl.G, N, N), **f32)
    # the public calls want one storage type per call, where the step's own
    # launches mix BF16 images with FP32 sinogram buffers: with BF16 storage
    # these stand-ins read BF16 copies instead
    q_t = qbuf if arm.tdt == torch.float32 else qbuf.to(arm.tdt)
    p_t = pbuf if arm.tdt == torch.float32 else pbuf.to(arm.tdt)
    gtot_t = gtot if arm.tdt == torch.float32 else gtot.to(arm.tdt)
    x2 = arm.x2.reshape(BG, N, N)
    gx3 = arm.gx3.reshape(BG, N, N)
    gx2 = arm.gx2.reshape(BG, N, N)
    z = arm.z.reshape(BG, N, N)
    fwd_jobs = [S.Job(arm.x1, arm.r, mc_idx, aux=arm.y), S.Job(x2, pbuf, sk_idx)]
    # the form the step's own A launch takes (band sums: two launches)
    fwd_sums = S.ei_fwd_form(p, wl.B, wl.G, mc_idx, sk_idx, arm.wl.per_sample) == 1
    wfwd = torch.empty(max(S.band_sums_workspace_size(p, fwd_jobs), 16), dtype=torch.uint8,
                       device="cuda")
    bpa_jobs = [S.Job(gx3, p_t, sk_idx)]
    wsum = torch.empty(max(S.band_sums_workspace_size(p, bpa_jobs), 16), dtype=torch.uint8,
                       device="cuda")
    ops = {
        "rotate": lambda: S.rotate(arm.x1, arm.g, out=arm.x2),
        "joseph_fwd(MC+EI)": ((lambda: S.proj_fwd_multi_ws(p, fwd_jobs, work=wfwd)) if fwd_sums
                              else (lambda: S.proj_fwd_multi(p, fwd_jobs))),
        "ramlak(fwd)": lambda: S.filter(p, pbuf, np.pi / m, out=qbuf),
        "backproject": lambda: S.backproject(p, q_t, sk_idx, out=z),
        "backproject_adj": lambda: S.backproject_adj_multi_ws(p, bpa_jobs, work=wsum),
        "ramlak(bwd)": lambda: S.filter(p, pbuf, np.pi / m, out=qbuf),
        "joseph_adj(MC+EI)": lambda: S.proj_adj_multi(
            p, [S.Job(arm.r, arm.gx1, mc_idx, alpha=-2.0 * arm.mc_scale / wl.B),
                S.Job(qbuf, gtot.reshape(BG, N, N), sk_idx, aux=gx2, beta=1.0)]),
        "rotate_adj": lambda: S.rotate_adj(gtot_t, arm.g, beta=1.0, out=arm.gx1),
    }
    return ops


def kernel_breakdown(S, arm, stream, reps=20):
    """Device time of every operator of one step (`breakdown_ops`): `reps`
    copies are captured in a CUDA graph and the replay is timed with CUDA
    events on the launching stream."""
    import torch
    ops = breakdown_ops(S, arm)
    times = {}
    with torch.cuda.stream(stream):
        for name, fn in ops.items():
            for _ in range(2):
                fn()
            stream.synchronize()
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=stream):
                for _ in range(reps):
                    fn()
            graph.replay()
            stream.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            graph.replay()
            e1.record(stream)
            stream.synchronize()
            times[name] = 1e3 * e0.elapsed_time(e1) / reps  # microseconds per launch
    return times


def joseph_samples(plan, n_img, m_angles_idx):
    """Algorithmic work of Joseph's projector: (ray, line) crossings whose
    interpolation taps touch the image, pos in (-1, N), counted in FP64."""
    N, nd = plan.N, plan.n_det
    total = 0
    h, D = 0.5 * (N - 1), 0.5 * (nd - 1)
    k = np.arange(nd) - D
    L = np.arange(N)
    for a in m_angles_idx:
        th = np.radians(plan.angles_deg[a])
        c, s = np.cos(th), np.sin(th)
        phi = plan.angles_deg[a] % 180.0
        if phi <= 45.0 or phi > 135.0:
            pos = (k[:, None] - (h - L[None, :]) * s) / c + h
        else:
            pos = h - (k[:, None] - (L[None, :] - h) * c) / s
        total += int(np.count_nonzero((pos > -1) & (pos < N)))
    return total * n_img


FLOPS_PER_SAMPLE = 7  # position, fraction, lerp (sub + fma), accumulate


def pixel_angles(plan, n_img, n_ang):
    return n_img * plan.N * plan.N * n_ang


def algorithmic_flops(plan, arm, name):
    """FP32 flops a kernel of the step must do at the least: 7 per
    interpolation sample of its operator (a Joseph crossing inside the image
    for A and A^T; a pixel x angle for B and B^T), 3 per (output, odd tap)
    pair for the filter."""
    wl = arm.wl
    idx = arm.idx.cpu().numpy()
    mc_idx = idx if wl.mc_sketched else np.arange(wl.views)
    m = len(idx)
    BG = wl.B * wl.G
    if name.startswith("joseph"):
        return FLOPS_PER_SAMPLE * (joseph_samples(plan, wl.B, mc_idx)
                                   + joseph_samples(plan, BG, idx))
    if name.startswith("backproject"):
        return FLOPS_PER_SAMPLE * pixel_angles(plan, BG, m)
    if name.startswith("ramlak"):
        nd = plan.n_det
        return 3.0 * BG * m * nd * (nd // 2)
    return None


def csrc_digest():
    import hashlib
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2411_05771_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        if f.endswith((".cu", ".cuh")):
            h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def measured_traffic(kernel):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, or
    None if the kernels have changed since it was captured."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(path):
        return None
    digest = csrc_digest()
    for line in open(path):
        parts = line.split()
        if len(parts) == 3 and parts[0] == kernel and parts[2] == digest:
            return float(parts[1])
    return None


SMEM_BYTES_PER_SAMPLE = 8   # two 4-byte taps per interpolation sample


def algorithmic_bytes(plan, arm, name):
    """Compulsory DRAM bytes of an operator kernel of the step: its input
    images or sinograms once, its outputs once (4-byte storage)."""
    wl = arm.wl
    N, nd, BG, B = plan.N, plan.n_det, wl.B * wl.G, wl.B
    m, mc_m = arm.m, arm.mc_m
    img, sino = 4 * N * N, 4 * nd
    if name.startswith("joseph_fwd"):      # x1, x2 in; r (+ y rows) and p out
        return (B + BG) * img + B * mc_m * sino * 2 + BG * m * sino
    if name.startswith("joseph_adj"):      # r, v in; g_x2 in, g_x1, g_tot out
        return (B * mc_m + BG * m) * sino + (BG + B + BG) * img
    if name.startswith("backproject_adj"):  # g_z in, sinogram out
        return BG * img + BG * m * sino
    if name.startswith("backproject"):      # filtered sinogram in, z out
        return BG * m * sino + BG * img
    if name.startswith("ramlak"):
        return 2 * BG * m * sino
    return None


def roofline_entry(plan, arm, bd, dom, roofs, peaks):
    """The roofline of kernel `dom`: t_roof = max(FP32 work / FMA rate,
    shared-memory tap bytes / shared-memory bandwidth, compulsory DRAM bytes
    / DRAM bandwidth), every rate measured on this GPU (skei_measure_roofs;
    DRAM: MEASURED_PEAKS.json's copy bandwidth where present); frac =
    t_roof / measured time, reported against the binding roof."""
    t = bd[dom] * 1e-6
    flops = algorithmic_flops(plan, arm, dom)
    samples = flops / FLOPS_PER_SAMPLE if flops and not dom.startswith("ramlak") else 0
    smem = SMEM_BYTES_PER_SAMPLE * samples
    dram = algorithmic_bytes(plan, arm, dom) or 0
    hbm = float(peaks.get("hbm_gbs", 0.0)) * 1e9 or roofs["dram_read_bytes"]
    times = {"fp32": (flops or 0) / roofs["fp32_flops"], "smem": smem / roofs["smem_bytes"],
             "hbm": dram / hbm}
    bound = max(times, key=times.get)
    unit_peak = {"fp32": (roofs["fp32_flops"] / 1e12, "TFLOP/s", (flops or 0) / t / 1e12),
                 "smem": (roofs["smem_bytes"] / 1e9, "GB/s", smem / t / 1e9),
                 "hbm": (hbm / 1e9, "GB/s", dram / t / 1e9)}
    peak, unit, achieved = unit_peak[bound]
    return {"bound": bound, "kernel": dom, "achieved": achieved, "peak": peak, "unit": unit,
            "frac": times[bound] / t, "traffic": measured_traffic(dom),
            "peak_source": "measured on this GPU: skei_measure_roofs (FP32 FMA chains, 16-byte "
                           "shared loads)" + ("; HBM: MEASURED_PEAKS.json copy bandwidth"
                                              if peaks.get("hbm_gbs") else
                                              "; DRAM: skei_measure_roofs streaming read"),
            "work": f"{FLOPS_PER_SAMPLE} flop and {SMEM_BYTES_PER_SAMPLE} shared-memory bytes "
                    "(two 4-byte taps) per interpolation sample; compulsory DRAM bytes: inputs "
                    "and outputs once",
            "launch_us": bd[dom],
            "roof_us": {k: round(v * 1e6, 3) for k, v in times.items()},
            "frac_by_roof": {k: round(v / t, 4) for k, v in times.items()}}


def cpu_oracle_steps(prob, n_steps, sketched):
    """The FP64 oracle (single-threaded C loops + numpy) on the same step."""
    import oracle as O
    angs = prob["angs"]
    y = prob["y"][None]
    x0 = O.fbp(y, angs, N_IMG)
    theta = np.zeros((N_IMG, N_IMG))
    mom = np.zeros_like(theta)
    vel = np.zeros_like(theta)
    idx_all, g_all = step_params(n_steps, SKETCHED if sketched else PLAIN)
    mcs = (N_VIEWS / SKETCH) if sketched else 1.0
    t0 = time.perf_counter()
    for s in range(n_steps):
        idx = idx_all[s] if sketched else None
        _, grad, _ = O.ttt_grad(theta, x0, y, angs, idx, idx, g_all[s], LAM, mcs)
        theta, mom, vel = O.adam_step(theta, grad, mom, vel, s + 1, lr=LR)
    return n_steps / (time.perf_counter() - t0)


def _oracle_worker(n_steps, barrier, queue):
    """One replica of the oracle's TTT run (a spawned process): set-up, then
    `n_steps` timed steps once every replica is ready."""
    prob = make_problem()
    barrier.wait()
    queue.put(n_steps / cpu_oracle_steps(prob, n_steps, True))


def cpu_replicas(n_steps, procs=None):
    """The FP64 oracle on every host core: `procs` (default: all cores)
    independent replicas of the sketched TTT step in spawned processes, one
    thread each, started together.  Returns (steps/s over all replicas =
    total steps / the slowest replica's time, processes)."""
    import multiprocessing as mp
    import oracle as O
    O.build()   # once, before the replicas load it
    procs = procs or os.cpu_count() or 1
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS",
                                            "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        ctx = mp.get_context("spawn")
        barrier, queue = ctx.Barrier(procs), ctx.Queue()
        ps = [ctx.Process(target=_oracle_worker, args=(n_steps, barrier, queue))
              for _ in range(procs)]
        for p_ in ps:
            p_.start()
        secs = []
        while len(secs) < procs:
            try:
                secs.append(queue.get(timeout=5))
            except Exception:   # queue.Empty: check that no replica died
                dead = [p_.exitcode for p_ in ps if p_.exitcode not in (None, 0)]
                if dead:
                    for p_ in ps:
                        p_.kill()
                    raise RuntimeError(f"oracle replica failed (exit codes {dead})")
        for p_ in ps:
            p_.join()
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return procs * n_steps / max(secs), procs


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n = args.steps if args.steps > 0 else 3
    n = max(1, min(n, 5))
    if args.warmup > 0:
        cpu_replicas(1)
    v, procs = cpu_replicas(n)
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT,
        "n_gpus": args.gpus, "steps": n, "warmup": min(args.warmup, 1),
        "ms_per_step": 1e3 / v, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": dict(workload_config(), arm="sketched"),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": procs, "kind": "oracle",
                         "sample": f"{procs} replicas (one per host core, one thread each) x "
                                   f"{n} sketched TTT steps at 512^2 (FP64 C oracle)"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# -------------------------------------------------------------- ranks
def whole_job(ms, steps, world, device):
    """Max of the timed interval over the ranks (each runs its own replica)
    and the whole-job throughput: the steps all ranks ran / that max."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    return ms_max, world * steps / (ms_max * 1e-3)


# ------------------------------------------------------------------ suite
def time_graph(fn, stream, reps=20):
    """Microseconds per call of `fn`: `reps` calls captured in a CUDA graph,
    one warm replay, one timed replay (CUDA events on the launching stream)."""
    import torch
    with torch.cuda.stream(stream):
        for _ in range(2):
            fn()
        stream.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            for _ in range(reps):
                fn()
        graph.replay()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        graph.replay()
        e1.record(stream)
        stream.synchronize()
    return 1e3 * e0.elapsed_time(e1) / reps


def fp32_peak(dev):
    import torch
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    sm = torch.cuda.get_device_properties(dev).multi_processor_count
    return sm * 128 * 2 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12


def op_line(workload, op, us, samples, peak, **extra):
    flops = FLOPS_PER_SAMPLE * samples
    line = {"suite": workload, "op": op, "us": round(us, 2), "samples": int(samples),
            "tflops": round(flops / (us * 1e-6) / 1e12, 3),
            "roofline_frac": round(flops / (us * 1e-6) / 1e12 / peak, 4)}
    line.update(extra)
    print(json.dumps(line), flush=True)


def ttt_bn_suite(S, dev, stream, channels=16, layers=4):
    """BN-only test-time training (Sec. 3.3) on the 512^2 workload: the
    residual CNN stand-in (frozen seeded 3x3 convolutions, cuDNN, FP32 without
    TF32; batch-statistics BN + ReLU in libskei) run twice per step around the
    operators, autograd backward through it, Adam on the BN parameters only;
    the whole step is one CUDA graph.  Sketched vs plain arm as in the
    headline (the draws of step 1)."""
    import torch
    from paper_2411_05771_gb300 import inputs as I
    from paper_2411_05771_gb300.autograd import skei_loss
    from paper_2411_05771_gb300.net import ResCNN
    saved = (torch.backends.cudnn.allow_tf32, torch.backends.cudnn.benchmark)
    torch.backends.cudnn.allow_tf32 = False
    torch.backends.cudnn.benchmark = True
    prob = make_problem(SKETCHED)
    plan = S.Plan(N_IMG, N_VIEWS, prob["angs"])
    f32 = dict(dtype=torch.float32, device=dev)
    y = torch.tensor(prob["y"], **f32)[None]
    x0 = S.fbp(plan, y)
    wts = I.cnn_weights(channels=channels, layers=layers, seed=0)
    # the BN kernels alone at the network's largest activation: the B G = 4
    # transformed images x 16 channels of 512^2
    hbm = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs", 6787.9)) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 6787.9
    v = torch.randn((SKETCHED.B * SKETCHED.G, channels, N_IMG, N_IMG), **f32)
    gv = torch.randn_like(v)
    sc, sh = torch.ones(channels, **f32), torch.zeros(channels, **f32)
    bo = torch.empty_like(v)
    wbn = torch.empty(S.bn_workspace_size(*v.shape[:2], N_IMG * N_IMG), dtype=torch.uint8,
                      device=dev)
    _, mu, rs = S.bn_act_fwd(v, sc, sh, out=bo, work=wbn)
    nbytes = v.numel() * 4
    for op, fn, traffic in (("BN+ReLU forward", lambda: S.bn_act_fwd(v, sc, sh, out=bo, work=wbn),
                             2 * nbytes),
                            ("BN+ReLU backward",
                             lambda: S.bn_act_bwd(v, gv, sc, sh, mu, rs, work=wbn), 3 * nbytes)):
        us = time_graph(fn, stream, reps=10)
        gbs = traffic / (us * 1e-6) / 1e9
        print(json.dumps({"suite": "bn-4x16x512x512", "op": op, "us": round(us, 2),
                          "algorithmic_bytes": traffic, "gb_per_s": round(gbs, 1),
                          "roofline_frac_hbm": round(gbs / hbm, 3),
                          "launches": 2}), flush=True)
    del v, gv, bo, wbn

    res = {}
    for tag, wl in (("sketched", SKETCHED), ("plain", PLAIN)):
        idx_all, g_all = step_params(1, wl)
        idx = None if not wl.sketched else torch.tensor(idx_all[0], dtype=torch.int32,
                                                         device=dev)
        mc_idx = idx if wl.mc_sketched else None
        g = torch.tensor(g_all[0], dtype=torch.float64, device=dev)
        net = ResCNN(wts, dev)
        m1, v1 = torch.zeros_like(net.bn), torch.zeros_like(net.bn)
        step_no = torch.ones((), dtype=torch.int32, device=dev)

        def step(net=net, idx=idx, mc_idx=mc_idx, g=g, m1=m1, v1=v1, wl=wl, step_no=step_no):
            loss = skei_loss(plan, net(x0), y, net, g, mc_idx, idx, LAM, wl.mc_scale)
            (gr,) = torch.autograd.grad(loss, [net.bn])
            with torch.no_grad():
                S.adam_step(net.bn.data, m1, v1, step_no, gr, lr=LR)

        res[tag] = time_graph(step, stream, reps=5)
        torch.backends.cudnn.allow_tf32 = True
        res[tag + "_tf32"] = time_graph(step, stream, reps=5)
        torch.backends.cudnn.allow_tf32 = False
    torch.backends.cudnn.allow_tf32, torch.backends.cudnn.benchmark = saved
    print(json.dumps({"suite": "ttt-bn-512x512-60views-sketch30-G4",
                      "network": f"residual CNN, {layers} 3x3 conv layers x {channels} "
                                 "channels, batch-statistics BN + ReLU, FP32 (no TF32)",
                      "adapted": f"BN scale/shift only ({wts.bn.size} parameters)",
                      "sketched_steps_per_s": round(1e6 / res["sketched"], 1),
                      "plain_steps_per_s": round(1e6 / res["plain"], 1),
                      "speedup": round(res["plain"] / res["sketched"], 3),
                      "tf32_network": {"sketched_steps_per_s": round(1e6 / res["sketched_tf32"], 1),
                                       "plain_steps_per_s": round(1e6 / res["plain_tf32"], 1),
                                       "speedup": round(res["plain_tf32"] / res["sketched_tf32"],
                                                        3)}}), flush=True)


def mri_suite(S, dev, stream, N=128, Nc=15, accel=4, G=1, mc=2):
    """Multi-coil MRI (Sec. 3.4, Algorithm 3) at 128^2, 15 coils, 4x
    undersampling: the operators' times, and the EI step (residual stand-in
    network, one rotation per step) with all 15 coils, with a random subset
    of `mc` coils per step (SkEI, subsampling sketch) and with the coil
    sketch of `mc` coils (C-SkEI: 15 PCA virtual coils, R = 1 kept, the rest
    mixed by a Rademacher block)."""
    import torch
    from paper_2411_05771_gb300 import inputs as I
    from paper_2411_05771_gb300.mri import CoilSketch, CskArm
    f32 = dict(dtype=torch.float32, device=dev)
    maps = torch.tensor(I.coil_maps(Nc, N), **f32)
    mask = torch.tensor(I.undersampling_mask(N, accel), **f32)
    x_gt = torch.tensor(I.complex_phantom(0, N), **f32)[None]
    y = S.mri_fwd(x_gt, maps, mask)
    dinv = S.mri_dinv(maps)
    x0 = S.mri_adj(y, maps, mask, dinv)
    k = torch.empty_like(y)
    xo = torch.empty_like(x0)
    w = torch.empty(S.mri_workspace_size(N, Nc, 1), dtype=torch.uint8, device=dev)
    ops = {"A (15 coils)": lambda: S.mri_fwd(x0, maps, mask, out=k, work=w),
           "A^H (15 coils)": lambda: S.mri_adj(y, maps, mask, out=xo, work=w),
           "A^dagger (15 coils)": lambda: S.mri_adj(y, maps, mask, dinv, out=xo, work=w)}
    op_us = {name: round(time_graph(fn, stream), 2) for name, fn in ops.items()}
    # arms
    rng = np.random.default_rng(0)
    g = torch.tensor(rng.uniform(0, 360, (1, G)), dtype=torch.float64, device=dev)
    res = {}
    full = CskArm(x0, y, maps, mask, dinv, G)
    full.g.copy_(g)
    res["EI (15 coils)"] = time_graph(full.step, stream)
    # SkEI: a random subset of mc coils, selected inside every step
    sel = np.zeros((mc, Nc), dtype=np.complex64)
    sel[np.arange(mc), rng.choice(Nc, mc, replace=False)] = 1.0
    Wsel = torch.tensor(sel, device=dev)
    maps_s = S.coil_mix(Wsel, maps[None])[0].contiguous()
    y_s = S.coil_mix(Wsel, y)
    dinv_s = S.mri_dinv(maps_s)
    sub = CskArm(x0, y_s, maps_s, mask, dinv_s, G)
    sub.g.copy_(g)

    def sk_step():
        S.coil_mix(Wsel, maps[None], out=maps_s[None])
        S.coil_mix(Wsel, y, out=y_s)
        S.mri_dinv(maps_s, out=dinv_s)
        sub.step()
    res[f"SkEI ({mc} of {Nc} coils)"] = time_graph(sk_step, stream)
    cs = CoilSketch(y, maps, Nc, 1, I.rademacher(rng, (mc - 1, Nc - 1)))
    csk = CskArm(x0, cs.y, cs.maps, mask, cs.dinv, G)
    csk.g.copy_(g)
    res[f"C-SkEI ({mc} sketched coils)"] = time_graph(csk.step, stream)
    base = res["EI (15 coils)"]
    print(json.dumps({"suite": f"mri-{N}x{N}-{Nc}coils-{accel}x", "op_us": op_us,
                      "step_us": {k_: round(v, 2) for k_, v in res.items()},
                      "steps_per_s": {k_: round(1e6 / v, 1) for k_, v in res.items()},
                      "speedup_vs_EI": {k_: round(base / v, 3) for k_, v in res.items()},
                      "network": "F(u) = u + theta", "G": G,
                      "launches_per_step": CskArm.launches_per_step}), flush=True)


def suite(S, dev, stream):
    """The measurements behind the per-workload table: single operators
    (64^2 with 60 views; 8 x 256^2 with 180 views, full and a 45-angle
    sketch), the differentiated EI step at 8 x 4 x 256^2 (MC term on all
    180 views, EI term on the sketch), and the 16-instance batch of 256^2 /
    512^2 instances with sketches of 45-360 angles."""
    import torch
    from paper_2411_05771_gb300 import inputs as I
    peak = fp32_peak(dev)
    for name, N, views, B, m in (("64x64-60views", 64, 60, 1, None),
                                 ("8x256x256-180views-363bins", 256, 180, 8, 45)):
        plan = S.Plan(N, views)
        x = torch.tensor(np.stack([I.rasterize(I.random_ellipses(b), N) for b in range(B)]),
                         dtype=torch.float32, device=dev)
        sets = [("full", None, np.arange(views))]
        if m:
            off = I.random_sketch_offset(np.random.default_rng(0), views, m)
            sk = I.sketch_indices(views, m, off)
            sets.append((f"sketch{m}", torch.tensor(sk, dtype=torch.int32, device=dev), sk))
        for tag, idx, idx_np in sets:
            mm = len(idx_np)
            y = S.proj_fwd(plan, x, idx)
            xo = torch.empty_like(x)
            yo = torch.empty_like(y)
            work = torch.empty(max(S.fbp_workspace_size(plan, S.F32, B, mm), 16),
                               dtype=torch.uint8, device=dev)
            js = joseph_samples(plan, B, idx_np)
            pa = pixel_angles(plan, B, mm)
            fj = [S.Job(x, yo, idx)]
            wsum = torch.empty(max(S.band_sums_workspace_size(plan, fj), 16), dtype=torch.uint8,
                               device=dev)
            ops = [("A", lambda: S.proj_fwd(plan, x, idx, out=yo), js),
                   ("A (band sums)", lambda: S.proj_fwd_multi_ws(plan, fj, work=wsum), js),
                   ("A^T", lambda: S.proj_adj(plan, y, idx, out=xo), js),
                   ("H", lambda: S.filter(plan, y, 1.0, out=yo), None),
                   ("B", lambda: S.backproject(plan, y, idx, out=xo), pa),
                   ("B^T", lambda: S.backproject_adj(plan, x, idx, out=yo), pa),
                   ("B^T (band sums)", lambda: S.backproject_adj_multi_ws(plan, fj, work=wsum),
                    pa),
                   ("FBP", lambda: S.fbp(plan, y, idx, out=xo, work=work), pa)]
            for op, fn, smp in ops:
                us = time_graph(fn, stream)
                if smp is None:
                    nd = plan.n_det
                    macs = B * mm * nd * (nd // 2)
                    print(json.dumps({"suite": name, "op": op, "angles": tag, "us": round(us, 2),
                                      "tflops": round(3.0 * macs / (us * 1e-6) / 1e12, 3),
                                      "roofline_frac": round(3.0 * macs / (us * 1e-6) / 1e12
                                                             / peak, 4)}), flush=True)
                else:
                    op_line(name, op, us, smp, peak, angles=tag, B=B)

    # the differentiated EI step, MC on all views, EI on a 45-angle sketch
    wl = Workload(N=256, views=180, m=45, G=4, B=8, mc_sketched=False, noisy=False)
    wp = Workload(N=256, views=180, m=180, G=4, B=8, mc_sketched=False, noisy=False, draw_m=45)
    prob = make_problem(wl)
    plan = S.Plan(256, 180, prob["angs"])
    ws = Workload(N=256, views=180, m=45, G=4, B=8, mc_sketched=False, noisy=False,
                  per_sample=True)
    # the MC term on the sketch too (Algorithm 2's form), shared or per measurement
    wm = Workload(N=256, views=180, m=45, G=4, B=8, mc_sketched=True, noisy=False)
    wmp = Workload(N=256, views=180, m=45, G=4, B=8, mc_sketched=True, noisy=False,
                   per_sample=True)
    res = {}
    for tag, w in (("sketched", wl), ("plain", wp), ("per_sample", ws), ("mc_sketched", wm),
                   ("mc_sketched_per_sample", wmp)):
        arm = Arm(S, plan, prob, w, "f32", dev)
        idx_all, g_all = step_params(1, w)
        arm.load_params(idx_all[0], g_all[0], 1)
        res[tag] = time_graph(arm.step, stream)
    print(json.dumps({"suite": "ei-step-8x4x256x256-180views-sketch45", "G": 4, "B": 8,
                      "mc": "all 180 views", "ei": "45-angle sketch",
                      "sketched_steps_per_s": round(1e6 / res["sketched"], 1),
                      "plain_steps_per_s": round(1e6 / res["plain"], 1),
                      "speedup": round(res["plain"] / res["sketched"], 3),
                      "operator_work_ratio_bound": 3.0}), flush=True)
    # Algorithm 1 over 8 measurements with a sketch each
    print(json.dumps({"suite": "ei-step-8x4x256x256-180views-sketch45-per-sample", "G": 4,
                      "B": 8, "mc": "all 180 views", "ei": "45-angle sketch per measurement",
                      "per_sample_steps_per_s": round(1e6 / res["per_sample"], 1),
                      "shared_sketch_steps_per_s": round(1e6 / res["sketched"], 1),
                      "plain_steps_per_s": round(1e6 / res["plain"], 1),
                      "speedup_vs_plain": round(res["plain"] / res["per_sample"], 3)}),
          flush=True)
    print(json.dumps({"suite": "ei-step-8x4x256x256-180views-sketch45-mc-sketched", "G": 4,
                      "B": 8, "mc": "the 45-angle sketch", "ei": "the same sketch",
                      "shared_sketch_steps_per_s": round(1e6 / res["mc_sketched"], 1),
                      "per_sample_steps_per_s": round(1e6 / res["mc_sketched_per_sample"], 1),
                      "plain_steps_per_s": round(1e6 / res["plain"], 1),
                      "speedup_vs_plain": round(res["plain"] / res["mc_sketched"], 3)}),
          flush=True)

    ttt_bn_suite(S, dev, stream)
    mri_suite(S, dev, stream)

    # Theorem 1 on an explicit 32^2, 100-view A (probe.theorem1)
    from paper_2411_05771_gb300.probe import theorem1
    plan32 = S.Plan(32, 100)
    v = torch.tensor(np.stack([I.rasterize(I.random_ellipses(s), 32) for s in range(8)]),
                     dtype=torch.float32, device=dev)
    res = theorem1(plan32, ns_list=(2, 5, 10, 20), v=v)
    print(json.dumps({"suite": "theorem1-32x32-100views", **{k: res[k] for k in
                      ("rank", "sigma_1", "sigma_k", "kappa")},
                      "sketches": [{k: (round(x, 5) if isinstance(x, float) else x)
                                    for k, x in it.items()} for it in res["sketches"]]}),
          flush=True)

    # 16 instances mixing 256^2 / 360 angles and 512^2 / 720 angles
    rng = np.random.default_rng(4)
    sizes = [(256, 360), (512, 720)] * 8
    ms = rng.choice([45, 90, 180, 360], size=16)
    plans = {k: S.Plan(*k) for k in set(sizes)}
    for dt in (torch.float32, torch.bfloat16):
        for opname in ("PROJ_FWD", "PROJ_ADJ", "FBP"):
            op = getattr(S, opname)
            items, singles, samples = [], [], 0
            for q, ((N, n), m) in enumerate(zip(sizes, ms)):
                p = plans[(N, n)]
                off = I.random_sketch_offset(np.random.default_rng(q), n, int(m))
                sk = I.sketch_indices(n, int(m), off)
                idx = torch.tensor(sk, dtype=torch.int32, device=dev)
                img = torch.randn((1, N, N), device=dev).to(dt)
                sino = torch.randn((1, int(m), p.n_det), device=dev).to(dt)
                inp, out = (img, torch.empty_like(sino)) if op == S.PROJ_FWD else \
                    (sino, torch.empty_like(img))
                items.append(S.BatchItem(p, inp, out, idx))
                if op == S.PROJ_FWD:
                    singles.append(lambda p=p, inp=inp, idx=idx, out=out:
                                   S.proj_fwd(p, inp, idx, out=out))
                    samples += joseph_samples(p, 1, sk)
                elif op == S.PROJ_ADJ:
                    singles.append(lambda p=p, inp=inp, idx=idx, out=out:
                                   S.proj_adj(p, inp, idx, out=out))
                    samples += joseph_samples(p, 1, sk)
                else:
                    singles.append(lambda p=p, inp=inp, idx=idx, out=out: S.fbp(p, inp, idx, out=out))
                    samples += pixel_angles(p, 1, int(m))
            batch = S.Batch(op, items)
            us_default = time_graph(batch.run, stream, reps=5)
            batch.tune(reps=3)
            us_tuned = time_graph(batch.run, stream, reps=5)
            us_single = time_graph(lambda: [f() for f in singles], stream, reps=5)
            op_line("batch-16-mixed-256-512", opname, us_tuned, samples, peak,
                    dtype="f32" if dt == torch.float32 else "bf16",
                    us_untuned=round(us_default, 2), us_16_single_launches=round(us_single, 2),
                    tuned=batch.info(batch.info(0)["phases"] - 1))


def main():
    args = parse()
    if args.impl == "reference":
        reference_arm(args)
        return
    import torch
    import torch.distributed as dist
    from paper_2411_05771_gb300 import build as B
    B.build()
    from paper_2411_05771_gb300 import skei as S

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        gpu_id = str(local)

    if args.suite:
        suite(S, dev, torch.cuda.Stream(device=dev))
        return
    prob = make_problem()
    plan = S.Plan(N_IMG, N_VIEWS, prob["angs"])
    if args.profile:
        arm = Arm(S, plan, prob, SKETCHED, args.dtype, dev)
        ops = breakdown_ops(S, arm)
        torch.cuda.synchronize()
        arm.step()
        arm.step()
        torch.cuda.synchronize()
        for fn in ops.values():
            fn()
        torch.cuda.synchronize()
        print(json.dumps({"profile_run": "ok", "launches_per_step": arm.launches_per_step,
                          "breakdown": list(ops)}))
        return
    sk = Arm(S, plan, prob, SKETCHED, args.dtype, dev)
    pl = Arm(S, plan, prob, PLAIN, "f32", dev)
    other = "bf16" if args.dtype == "f32" else "f32"
    sk2 = Arm(S, plan, prob, SKETCHED, other, dev)

    # reconstruction quality: both arms, same start, same draws
    curve_sk = psnr_curve(sk, prob["x_gt"], PSNR_ITERS)
    curve_pl = psnr_curve(pl, prob["x_gt"], PSNR_ITERS)
    curve_sk2 = psnr_curve(sk2, prob["x_gt"], PSNR_ITERS)

    K_req, W = args.steps, max(args.warmup, 3)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)

    def estimate_ms(arm):
        """Device time of one graph-replayed step (a short untimed probe),
        used to size the timed region to at least MIN_TIMED_S."""
        arm.reset()
        us = time_graph(arm.step, stream, reps=20)
        arm.reset()
        return 1e-3 * us

    # the timed region lasts at least MIN_TIMED_S of device time, so that
    # the clock record has samples whatever --steps is; `steps` reports the
    # steps actually timed
    K = max(K_req, min(MAX_TIMED_STEPS, int(np.ceil(1e3 * MIN_TIMED_S / estimate_ms(pl)))),
            min(MAX_TIMED_STEPS, int(np.ceil(1e3 * MIN_TIMED_S / estimate_ms(sk)))))

    def timed(arm):
        """Device time of K graph-replayed steps.  The draws of all W + K
        steps (sketch rows, rotation angles, step numbers) are inputs,
        resident before the timed region as one table; the step graph's
        first kernel loads its row (skei_step_draws)."""
        arm.reset()
        idx_all, g_all = step_params(W + K, arm.wl, first=PSNR_ITERS + 1)
        with torch.cuda.stream(stream):
            for s in range(2):  # warm the library's one-time setup before capture
                arm.step()
            table = torch.from_numpy(arm.pack_params(idx_all, g_all, 1)).to(dev)
            counter = torch.zeros(1, dtype=torch.int32, device=dev)
            stream.synchronize()
            graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(graph, stream=stream):
                S.step_draws(table, counter, arm.params)
                arm.step()
            arm.reset()
            counter.zero_()

            def one(s):
                graph.replay()

            for s in range(W):
                flush.zero_()
                one(s)
            stream.synchronize()
            if world > 1:
                dist.barrier()
            torch.cuda.synchronize()
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(K)]
            clocks = Clocks(gpu_id)
            t_wall = time.perf_counter()
            for s in range(K):
                flush.zero_()  # L2 flush outside the timed interval
                evs[s][0].record(stream)
                one(W + s)
                evs[s][1].record(stream)
            stream.synchronize()
            t_wall = time.perf_counter() - t_wall
            clk = clocks.stop()
            torch.cuda.synchronize()
            if counter.item() != W + K:
                raise RuntimeError(f"step draws: counter {counter.item()} after {W + K} steps")
            if world > 1:
                dist.barrier()
        dev_ms = sum(a.elapsed_time(b) for a, b in evs)
        return dev_ms, t_wall, clk

    sk_ms, sk_wall, clk = timed(sk)
    pl_ms, pl_wall, clk_pl = timed(pl)
    sk2_ms, _, clk2 = timed(sk2)

    # end to end through the public API (eager calls from Python), with the
    # measurement copied host->device and the loss read back every step
    host_y = torch.from_numpy(prob["y"][None].astype(np.float32)).pin_memory()
    if sk.tdt != torch.float32:
        host_y = host_y.to(sk.tdt).pin_memory()
    host_loss = torch.empty(1, dtype=torch.float64).pin_memory()
    idx_all, g_all = step_params(K, SKETCHED, first=PSNR_ITERS + 1 + W + K)
    h_par = torch.from_numpy(sk.pack_params(idx_all, g_all, 1)).pin_memory()
    sk.reset()
    with torch.cuda.stream(stream):
        for s in range(W):
            sk.y.copy_(host_y, non_blocking=True)
            sk.step()
        stream.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for s in range(K):
            sk.y.copy_(host_y, non_blocking=True)
            sk.params.copy_(h_par[s], non_blocking=True)
            sk.step()
            host_loss.copy_(sk.loss, non_blocking=True)
        e1.record(stream)
        stream.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    h2d = host_y.numel() * host_y.element_size() + sk.param_bytes
    d2h = 8

    # per-kernel device times and the roofline of the dominant kernel, on
    # roofs measured on this GPU
    bd = kernel_breakdown(S, sk, stream)
    dom = max(bd, key=bd.get)
    with torch.cuda.stream(stream):
        roofs = S.measure_roofs()
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    roof = roofline_entry(plan, sk, bd, dom, roofs, peaks)
    kernels = {}
    for k, v in bd.items():
        kernels[k] = {"us": round(v, 2)}
        if algorithmic_flops(plan, sk, k):
            e = roofline_entry(plan, sk, bd, k, roofs, peaks)
            kernels[k].update(bound=e["bound"], frac=round(e["frac"], 4),
                              tflops=round(algorithmic_flops(plan, sk, k) / (v * 1e-6) / 1e12, 3))

    sk_ms_max, value = whole_job(sk_ms, K, world, dev)

    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline:
            n_cpu = args.cpu_steps or 2
            v, procs = cpu_replicas(n_cpu)
            cpu = {"value": v, "unit": UNIT, "cores": procs, "kind": "oracle",
                   "sample": f"{procs} replicas (one per host core, one thread each) x {n_cpu} "
                             "sketched TTT steps at 512^2 (FP64 C oracle)"}
        line = {
            "metric": METRIC,
            "value": value,
            "unit": UNIT,
            "n_gpus": world,
            "steps": K,
            "warmup": W,
            "ms_per_step": sk_ms_max / K,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": args.dtype,
            "data": "synthetic",
            "config": dict(workload_config(), graph=True,
                           l2="flushed between timed steps (256 MiB write, untimed)",
                           draws="all steps' draws resident; each step's graph loads its row"),
            "steps_requested": K_req,
            "plain": {"value": K / (pl_ms * 1e-3), "ms_per_step": pl_ms / K, "dtype": "f32",
                      "clocks": clk_pl},
            "speedup_vs_plain": pl_ms / sk_ms,
            "psnr": psnr_block(curve_sk, curve_pl, sk_ms / K, pl_ms / K),
            f"sketched_{other}": {
                "value": K / (sk2_ms * 1e-3), "ms_per_step": sk2_ms / K, "dtype": other,
                "storage": "images and sinograms in BF16, FP32 arithmetic" if other == "bf16"
                else "FP32", "speedup_vs_plain": pl_ms / sk2_ms, "clocks": clk2,
                "psnr": {k: v for k, v in psnr_block(curve_sk2, curve_pl, sk2_ms / K,
                                                     pl_ms / K).items()
                         if k in ("at_ref_iters", "to_plain_ref", "to_plain_best",
                                  "sketched_best")}},
            "e2e": {"value": K / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": (sk.launches_per_step + 1) * K,   # + the draws kernel
            "roofline": roof,
            "roofs_measured": {"fp32_tflops": roofs["fp32_flops"] / 1e12,
                               "smem_gbs": roofs["smem_bytes"] / 1e9,
                               "l2_gbs": roofs["l2_bytes"] / 1e9,
                               "dram_read_gbs": roofs["dram_read_bytes"] / 1e9, "sms": roofs["sms"]},
            "kernels": kernels,
            "clocks": clk,
            "cpu_baseline": cpu,
            "wall_s_timed": sk_wall,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
