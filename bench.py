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


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="skei", choices=["skei", "reference"])
    ap.add_argument("--dtype", default="f32", choices=["f32", "bf16"],
                    help="storage type of the sketched arm")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-steps", type=int, default=0, help="oracle steps (0 = auto, ~15 s)")
    ap.add_argument("--profile", action="store_true",
                    help="set up the sketched arm, run one warm and one more step, and exit "
                         "(a short, untimed run for ncu: 2 launches of set-up, then 13 per step)")
    return ap.parse_args()


# --------------------------------------------------------------------- inputs
def make_problem(seed=0):
    from paper_2411_05771_gb300 import inputs as I
    e = I.random_ellipses(seed)
    x_gt = I.rasterize(e, N_IMG)
    angs = I.uniform_angles(N_VIEWS)
    n_det = int(np.ceil(N_IMG * np.sqrt(2.0))) | 1
    y_clean = I.analytic_sinogram(e, N_IMG, angs, n_det)
    y = I.noisy_sinogram(y_clean, N_IMG, seed=seed + 77)
    return dict(x_gt=x_gt, angs=angs, n_det=n_det, y=y)


def step_params(n_steps, sketched, first=0):
    from paper_2411_05771_gb300 import inputs as I
    idx, g = [], []
    for s in range(first, first + n_steps):
        rng = I.step_rng(s)
        off = I.random_sketch_offset(rng, N_VIEWS, SKETCH)
        idx.append(I.sketch_indices(N_VIEWS, SKETCH, off) if sketched
                   else np.arange(N_VIEWS, dtype=np.int32))
        g.append(I.rotation_angles(rng, BATCH, G_ROT))
    return np.stack(idx).astype(np.int32), np.stack(g)


# ------------------------------------------------------------------ GPU arm
class Arm:
    """One TTT problem on the GPU with all buffers resident; `step()` issues
    Algorithm 2's iteration through the C ABI on the current stream."""

    def __init__(self, S, plan, prob, sketched, dtype, device):
        import torch
        self.S, self.plan, self.sketched = S, plan, sketched
        self.tdt = torch.float32 if dtype == "f32" else torch.bfloat16
        N, nd = N_IMG, plan.n_det
        self.m = SKETCH if sketched else N_VIEWS
        self.mc_scale = (N_VIEWS / SKETCH) if sketched else 1.0
        d = device
        self.y = torch.tensor(prob["y"][None], dtype=self.tdt, device=d)
        y32 = torch.tensor(prob["y"][None], dtype=torch.float32, device=d)
        self.x0 = S.fbp(plan, y32).to(self.tdt).contiguous()
        self.theta = torch.zeros((N, N), dtype=torch.float32, device=d)
        self.m1 = torch.zeros_like(self.theta)
        self.v1 = torch.zeros_like(self.theta)
        self.step_no = torch.zeros(1, dtype=torch.int32, device=d)
        self.idx = torch.zeros(self.m, dtype=torch.int32, device=d)
        self.g = torch.zeros((BATCH, G_ROT), dtype=torch.float64, device=d)
        self.x1 = torch.empty((BATCH, N, N), dtype=self.tdt, device=d)
        self.r = torch.empty((BATCH, self.m, nd), dtype=self.tdt, device=d)
        self.x2 = torch.empty((BATCH, G_ROT, N, N), dtype=self.tdt, device=d)
        self.z = torch.empty_like(self.x2)
        self.x3 = torch.empty_like(self.x2)
        self.gx2 = torch.empty_like(self.x2)
        self.gx3 = torch.empty_like(self.x2)
        self.gx1 = torch.empty_like(self.x1)
        self.loss = torch.empty(1, dtype=torch.float64, device=d)
        self.mc = torch.empty(BATCH, dtype=torch.float64, device=d)
        self.ei = torch.empty((BATCH, G_ROT), dtype=torch.float64, device=d)
        code = S.F32 if dtype == "f32" else S.BF16
        self.work = torch.empty(max(S.ei_workspace_size(plan, code, BATCH, G_ROT, self.m, self.m),
                                    16), dtype=torch.uint8, device=d)
        idx_all, g_all = step_params(1, sketched)
        self.load_params(idx_all[0], g_all[0], 1)

    def load_params(self, idx, g, step_no):
        import torch
        self.idx.copy_(torch.as_tensor(idx))
        self.g.copy_(torch.as_tensor(g))
        self.step_no.fill_(step_no)

    def step(self):
        S, p = self.S, self.plan
        mc_idx = self.idx if self.sketched else None
        sk_idx = self.idx if self.sketched else None
        S.residual_add(self.x0, self.theta, out=self.x1)                      # x1 = F(x0)
        S.ei_loss_fwd(p, self.x1, self.y, self.g, mc_idx, sk_idx, work=self.work,
                      out=(self.r, self.x2, self.z))
        S.residual_add(self.z, self.theta, out=self.x3)                       # x3 = F(z)
        S.ei_loss_finish(self.x2, self.x3, self.r, LAM, self.mc_scale, work=self.work,
                         out=(self.loss, self.mc, self.ei, self.gx2, self.gx3))
        S.ei_loss_bwd(p, self.r, self.gx2, self.gx3, self.g, self.mc_scale / BATCH, mc_idx,
                      sk_idx, work=self.work, out=self.gx1)
        # dL/dtheta = dL/dx1 + sum_g dL/dx3 (F's Jacobian is the identity)
        S.adam_step(self.theta, self.m1, self.v1, self.step_no, self.gx1, self.gx3, lr=LR)

    launches_per_step = 13  # 1 + 4 + 1 + 2 + 4 + 1 kernels, see step()

    def reset(self):
        self.theta.zero_()
        self.m1.zero_()
        self.v1.zero_()


def psnr_curve(arm, x_gt, iters, every=25):
    """Algorithm 2 for `iters` iterations from theta = 0; PSNR of F(x0) =
    x0 + theta against the phantom every `every` iterations (untimed)."""
    import torch
    arm.reset()
    idx_all, g_all = step_params(iters, arm.sketched)
    rngv = float(x_gt.max() - x_gt.min())
    curve = {}
    for s in range(iters + 1):
        if s % every == 0:
            torch.cuda.synchronize()
            rec = (arm.x0.double() + arm.theta.double()).cpu().numpy()[0]
            curve[s] = 10 * np.log10(rngv * rngv / float(np.mean((rec - x_gt) ** 2)))
        if s == iters:
            break
        arm.load_params(idx_all[s], g_all[s], s + 1)
        arm.step()
    return curve


def psnr_block(c_sk, c_pl, ms_sk, ms_pl):
    """Equal-PSNR comparison: the sketched arm's time to reach the plain
    arm's PSNR after PSNR_REF_ITERS iterations, and to reach the plain arm's
    best PSNR over the whole trajectory."""
    ref = c_pl[PSNR_REF_ITERS]
    best_it = max(c_pl, key=c_pl.get)
    best = c_pl[best_it]
    out = {"iters_run": PSNR_ITERS, "fbp_x0": c_pl[0],
           "at_ref_iters": {"iters": PSNR_REF_ITERS, "plain": ref, "sketched": c_sk[PSNR_REF_ITERS],
                            "delta_db": c_sk[PSNR_REF_ITERS] - ref},
           "plain_best": {"psnr": best, "iters": best_it},
           "sketched_final": c_sk[max(c_sk)]}
    for key, target, it_pl in (("to_plain_ref", ref, PSNR_REF_ITERS), ("to_plain_best", best, best_it)):
        it_sk = iters_to_reach(c_sk, target)
        if it_sk is None:
            out[key] = {"target_db": target, "sketched_iters": None}
            continue
        t_pl, t_sk = it_pl * ms_pl, it_sk * ms_sk
        out[key] = {"target_db": target, "plain_iters": it_pl, "sketched_iters": it_sk,
                    "plain_ms": t_pl, "sketched_ms": t_sk, "speedup": t_pl / t_sk}
    out["curve_every_100"] = {"plain": {k: round(v, 3) for k, v in c_pl.items() if k % 100 == 0},
                              "sketched": {k: round(v, 3) for k, v in c_sk.items() if k % 100 == 0}}
    return out


def iters_to_reach(curve, target):
    """First iteration (linearly interpolated between samples) at which the
    curve reaches `target`, or None."""
    its = sorted(curve)
    for a, b in zip(its, its[1:]):
        if curve[a] >= target:
            return float(a)
        if curve[b] >= target:
            return a + (b - a) * (target - curve[a]) / (curve[b] - curve[a])
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
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

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
        for line in open(self.path):
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


def kernel_breakdown(S, arm, stream, reps=20):
    """Device time of every kernel launch of one step, each re-issued with
    the step's own arguments: `reps` copies are captured in a CUDA graph and
    the replay is timed with CUDA events on the launching stream."""
    import torch
    p = arm.plan
    mc_idx = arm.idx if arm.sketched else None
    sk_idx = arm.idx if arm.sketched else None
    BG, m = BATCH * G_ROT, arm.m
    f32 = dict(dtype=torch.float32, device="cuda")
    pbuf = torch.empty((BG, m, p.n_det), **f32)
    qbuf = torch.empty_like(pbuf)
    gtot = torch.empty((BATCH, G_ROT, N_IMG, N_IMG), **f32)
    # the public calls want one storage type per call, where the step's own
    # launches mix BF16 images with FP32 sinogram buffers: with BF16 storage
    # these stand-ins read BF16 copies instead
    q_t = qbuf if arm.tdt == torch.float32 else qbuf.to(arm.tdt)
    p_t = pbuf if arm.tdt == torch.float32 else pbuf.to(arm.tdt)
    gtot_t = gtot if arm.tdt == torch.float32 else gtot.to(arm.tdt)
    x2 = arm.x2.reshape(BG, N_IMG, N_IMG)
    gx3 = arm.gx3.reshape(BG, N_IMG, N_IMG)
    gx2 = arm.gx2.reshape(BG, N_IMG, N_IMG)
    z = arm.z.reshape(BG, N_IMG, N_IMG)
    ops = {
        "residual_add(x1)": lambda: S.residual_add(arm.x0, arm.theta, out=arm.x1),
        "rotate": lambda: S.rotate(arm.x1, arm.g, out=arm.x2),
        "joseph_fwd(MC+EI)": lambda: S.proj_fwd_multi(
            p, [S.Job(arm.x1, arm.r, mc_idx, aux=arm.y), S.Job(x2, pbuf, sk_idx)]),
        "ramlak(fwd)": lambda: S.filter(p, pbuf, np.pi / m, out=qbuf),
        "backproject": lambda: S.backproject(p, q_t, sk_idx, out=z),
        "residual_add(x3)": lambda: S.residual_add(arm.z, arm.theta, out=arm.x3),
        "loss_finish": lambda: S.ei_loss_finish(
            arm.x2, arm.x3, arm.r, LAM, arm.mc_scale, work=arm.work,
            out=(arm.loss, arm.mc, arm.ei, arm.gx2, arm.gx3)),
        "backproject_adj": lambda: S.backproject_adj(p, gx3, sk_idx, out=p_t),
        "ramlak(bwd)": lambda: S.filter(p, pbuf, np.pi / m, out=qbuf),
        "joseph_adj(MC+EI)": lambda: S.proj_adj_multi(
            p, [S.Job(arm.r, arm.gx1, mc_idx, alpha=-2.0 * arm.mc_scale / BATCH),
                S.Job(qbuf, gtot.reshape(BG, N_IMG, N_IMG), sk_idx, aux=gx2, beta=1.0)]),
        "rotate_adj": lambda: S.rotate_adj(gtot_t, arm.g, beta=1.0, out=arm.gx1),
        "adam": lambda: S.adam_step(arm.theta, arm.m1, arm.v1, arm.step_no, arm.gx1, arm.gx3,
                                    lr=LR),
    }
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
    """FP32 flops a kernel of the step must do at the least: 7 per nonzero
    of its operator (Joseph crossings inside the image for A and A^T; pixel
    x angle for B and B^T), 3 per (output, odd tap) pair for the filter."""
    idx = arm.idx.cpu().numpy()
    m = len(idx)
    BG = BATCH * G_ROT
    if name.startswith("joseph"):
        return FLOPS_PER_SAMPLE * (joseph_samples(plan, BATCH, idx)
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


def roofline_entry(plan, arm, bd, dom, dev):
    import torch
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    work = algorithmic_flops(plan, arm, dom)
    if not work:
        return {"bound": "hbm", "kernel": dom, "achieved": None, "peak": peaks.get("hbm_gbs"),
                "unit": "GB/s", "frac": None, "traffic": measured_traffic(dom)}
    peak = sm_count * 128 * 2 * max_mhz * 1e6 / 1e12
    achieved = work / (bd[dom] * 1e-6) / 1e12
    return {"bound": "alu", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": measured_traffic(dom),
            "peak_source": f"derived: {sm_count} SMs x 128 FP32 lanes x 2 flop x {max_mhz:.0f} MHz",
            "work": f"{FLOPS_PER_SAMPLE} flop per operator nonzero", "launch_us": bd[dom]}


def cpu_oracle_steps(prob, n_steps, sketched):
    """The FP64 oracle (single-threaded C loops + numpy) on the same step."""
    import oracle as O
    angs = prob["angs"]
    y = prob["y"][None]
    x0 = O.fbp(y, angs, N_IMG)
    theta = np.zeros((N_IMG, N_IMG))
    mom = np.zeros_like(theta)
    vel = np.zeros_like(theta)
    idx_all, g_all = step_params(n_steps, sketched)
    mcs = (N_VIEWS / SKETCH) if sketched else 1.0
    t0 = time.perf_counter()
    for s in range(n_steps):
        idx = idx_all[s] if sketched else None
        _, grad, _ = O.ttt_grad(theta, x0, y, angs, idx, idx, g_all[s], LAM, mcs)
        theta, mom, vel = O.adam_step(theta, grad, mom, vel, s + 1, lr=LR)
    return n_steps / (time.perf_counter() - t0)


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    prob = make_problem()
    n = args.steps if args.steps > 0 else 3
    n = max(1, min(n, 5))
    for _ in range(min(args.warmup, 1)):
        cpu_oracle_steps(prob, 1, True)
    v = cpu_oracle_steps(prob, n, True)
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT,
        "n_gpus": args.gpus, "steps": n, "warmup": min(args.warmup, 1),
        "ms_per_step": 1e3 / v, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "ttt-512x512-60views-725bins-sketch30-G4", "arm": "sketched"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{n} sketched TTT steps at 512^2 (FP64 C oracle, 1 thread)"},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


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

    prob = make_problem()
    plan = S.Plan(N_IMG, N_VIEWS, prob["angs"])
    if args.profile:
        arm = Arm(S, plan, prob, True, args.dtype, dev)
        arm.step()
        arm.step()
        torch.cuda.synchronize()
        print(json.dumps({"profile_run": "ok", "launches": 2 + 2 * Arm.launches_per_step}))
        return
    sk = Arm(S, plan, prob, True, args.dtype, dev)
    pl = Arm(S, plan, prob, False, "f32", dev)

    # reconstruction quality: both arms, same start, same draws
    curve_sk = psnr_curve(sk, prob["x_gt"], PSNR_ITERS)
    curve_pl = psnr_curve(pl, prob["x_gt"], PSNR_ITERS)

    K, W = args.steps, max(args.warmup, 3)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)
    stream = torch.cuda.Stream(device=dev)

    def timed(arm, use_graph):
        arm.reset()
        idx_all, g_all = step_params(W + K, arm.sketched, first=PSNR_ITERS + 1)
        with torch.cuda.stream(stream):
            graph = None
            if use_graph:
                for s in range(2):  # warm the library's one-time setup before capture
                    arm.step()
                stream.synchronize()
                graph = torch.cuda.CUDAGraph()
                with torch.cuda.graph(graph, stream=stream):
                    arm.step()
            host_idx = torch.from_numpy(idx_all).pin_memory()
            host_g = torch.from_numpy(g_all).pin_memory()
            host_step = torch.arange(1, W + K + 1, dtype=torch.int32).pin_memory()

            def one(s):
                arm.idx.copy_(host_idx[s], non_blocking=True)
                arm.g.copy_(host_g[s], non_blocking=True)
                arm.step_no.copy_(host_step[s:s + 1], non_blocking=True)
                if graph is not None:
                    graph.replay()
                else:
                    arm.step()

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
            if world > 1:
                dist.barrier()
        dev_ms = sum(a.elapsed_time(b) for a, b in evs)
        return dev_ms, t_wall, clk

    sk_ms, sk_wall, clk = timed(sk, True)
    pl_ms, _, _ = timed(pl, True)

    # end to end through the public API (eager calls from Python), with the
    # measurement copied host->device and the loss read back every step
    host_y = torch.from_numpy(prob["y"][None].astype(np.float32)).pin_memory()
    if sk.tdt != torch.float32:
        host_y = host_y.to(sk.tdt).pin_memory()
    host_loss = torch.empty(1, dtype=torch.float64).pin_memory()
    idx_all, g_all = step_params(K, True, first=PSNR_ITERS + 1 + W + K)
    h_idx = torch.from_numpy(idx_all).pin_memory()
    h_g = torch.from_numpy(g_all).pin_memory()
    h_step = torch.arange(1, K + 1, dtype=torch.int32).pin_memory()
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
            sk.idx.copy_(h_idx[s], non_blocking=True)
            sk.g.copy_(h_g[s], non_blocking=True)
            sk.step_no.copy_(h_step[s:s + 1], non_blocking=True)
            sk.step()
            host_loss.copy_(sk.loss, non_blocking=True)
        e1.record(stream)
        stream.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    h2d = host_y.numel() * host_y.element_size() + h_idx[0].numel() * 4 + h_g[0].numel() * 8 + 4
    d2h = 8

    # per-kernel device times and the roofline of the dominant kernel
    bd = kernel_breakdown(S, sk, stream)
    dom = max(bd, key=bd.get)
    roof = roofline_entry(plan, sk, bd, dom, dev)
    kernels = {k: {"us": round(v, 2)} for k, v in bd.items()}
    for k in kernels:
        w = algorithmic_flops(plan, sk, k)
        if w:
            kernels[k]["tflops"] = round(w / (bd[k] * 1e-6) / 1e12, 3)

    total_ms = torch.tensor([sk_ms], dtype=torch.float64, device=dev)
    if world > 1:
        dist.all_reduce(total_ms, op=dist.ReduceOp.MAX)
    sk_ms_max = float(total_ms.item())

    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline:
            n_cpu = args.cpu_steps or 6
            v = cpu_oracle_steps(prob, n_cpu, True)
            cpu = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                   "sample": f"{n_cpu} sketched TTT steps at 512^2 (FP64 C oracle, 1 thread)"}
        line = {
            "metric": METRIC,
            "value": world * K / (sk_ms_max * 1e-3),
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
            "config": {"workload": "ttt-512x512-60views-725bins-sketch30-G4",
                       "N": N_IMG, "views": N_VIEWS, "n_det": plan.n_det, "sketch": SKETCH,
                       "G": G_ROT, "B": BATCH, "lambda": LAM, "network": "F(u)=u+theta",
                       "optimizer": "adam lr 5e-4", "graph": True,
                       "l2": "flushed between timed steps (256 MiB write, untimed)"},
            "plain": {"value": K / (pl_ms * 1e-3), "ms_per_step": pl_ms / K, "dtype": "f32"},
            "speedup_vs_plain": pl_ms / sk_ms,
            "psnr": psnr_block(curve_sk, curve_pl, sk_ms / K, pl_ms / K),
            "e2e": {"value": K / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": d2h},
            "gpu_launches": Arm.launches_per_step * K,
            "roofline": roof,
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
