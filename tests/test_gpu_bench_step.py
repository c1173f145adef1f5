"""Parity of the step the benchmark times, at the benchmark's own size and
launch forms, against the FP64 oracle.

The step is Algorithm 2's iteration on the 512^2 test-time-training workload
(Eq. (e:skeilossttt)): 60 views x 725 bins, a 30-angle interleaved sketch
that both the MC term (scaled by n/m = 2) and the EI term use, G = 4
rotations, B = 1, the stand-in network F(u) = u + theta and Adam.  It is
built exactly as bench.py builds it (its Arm class: the same buffers, the
same entry points, hence the same launch forms: the band sums of A with the
MC image riding in the EI group's CTAs, B and A^T over one group of 4 with
the launch's own tile height, B^T's band sums), run eagerly and as one
replay of the captured CUDA graph, in FP32 and with BF16 storage.

Every stored result is compared element by element with the oracle on the
same inputs: r, x2, z, x3, the loss and its parts, g_x2, g_x1 and the
Adam-updated theta (from a non-trivial Adam state, so that the update
depends on the gradient's values, not only on its signs)."""
import numpy as np
import pytest
import torch

import bench as BN
import oracle as O

pytestmark = pytest.mark.gpu

# FP32: rel-L2 <= 1e-5; BF16 storage with FP32 arithmetic: rel-L2 <= 1e-2
# against the oracle on the BF16-rounded inputs (x1, y)
TOL = {"f32": 1e-5, "bf16": 1e-2}


@pytest.fixture(scope="module")
def S():
    from paper_2411_05771_gb300 import skei
    return skei


@pytest.fixture(scope="module")
def prob():
    return BN.make_problem()


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def host(t):
    return t.detach().double().cpu().numpy()


def _state(N, seed=5):
    """A mid-run Adam state: theta, first and second moments, step 7."""
    rng = np.random.default_rng(seed)
    theta = 0.01 * rng.standard_normal((N, N))
    m1 = 1e-4 * rng.standard_normal((N, N))
    v1 = (1e-4 * rng.standard_normal((N, N))) ** 2
    return theta.astype(np.float32), m1.astype(np.float32), v1.astype(np.float32), 7


def _arm(S, prob, dtype):
    plan = S.Plan(BN.N_IMG, BN.N_VIEWS, prob["angs"])
    arm = BN.Arm(S, plan, prob, BN.SKETCHED, dtype, torch.device("cuda"))
    idx_all, g_all = BN.step_params(1, BN.SKETCHED, first=3)
    theta, m1, v1, step_no = _state(BN.N_IMG)
    return arm, idx_all[0], g_all[0], (theta, m1, v1, step_no)


def _load(arm, idx, g, st):
    theta, m1, v1, step_no = st
    arm.theta.copy_(torch.from_numpy(theta))
    arm.m1.copy_(torch.from_numpy(m1))
    arm.v1.copy_(torch.from_numpy(v1))
    arm.load_params(idx, g, step_no)


def _outputs(arm):
    torch.cuda.synchronize()
    return {k: getattr(arm, k).detach().clone() for k in
            ("x1", "r", "x2", "z", "x3", "gx2", "gx3", "gx1", "loss", "mc", "ei", "theta",
             "m1", "v1")}


def _oracle(prob, out, idx, g, st):
    """The FP64 oracle on the step's inputs: x1 as stored (x0 + theta,
    rounded to the storage type), the measurement as stored, the draws and
    the Adam state."""
    theta, m1, v1, step_no = (np.asarray(a, dtype=np.float64) if i < 3 else a
                              for i, a in enumerate(st))
    wl = BN.SKETCHED
    x1 = host(out["x1"])
    y = out["y"]
    angs = prob["angs"]
    r, x2, z = O.ei_stage1(x1, y, angs, idx, idx, g)
    x3 = z + theta[None, None]
    loss, mc, ei, gx2, gx3 = O.ei_finish(x2, x3, r, BN.LAM, wl.mc_scale)
    gx1 = O.ei_backward(r, gx2, gx3, angs, idx, idx, g, wl.mc_scale)
    grad = gx1.sum(axis=0) + gx3.sum(axis=(0, 1))
    return dict(r=r, x2=x2, z=z, x3=x3, loss=loss, mc=mc, ei=ei, gx2=gx2, gx1=gx1, grad=grad,
                y_mc=np.asarray(y)[:, idx], adam=(theta, m1, v1, step_no))


def _compare(out, ref, tol):
    errs = {
        # the residual's rounding is bounded by its operands: relative to y_S
        "r": float(np.linalg.norm(host(out["r"]) - ref["r"]) / np.linalg.norm(ref["y_mc"])),
        "x2": rel(host(out["x2"]), ref["x2"]),
        "z": rel(host(out["z"]), ref["z"]),
        "x3": rel(host(out["x3"]), ref["x3"]),
        "loss": abs(out["loss"].item() - ref["loss"]) / abs(ref["loss"]),
        "mc": rel(host(out["mc"]), ref["mc"]),
        "ei": rel(host(out["ei"]), ref["ei"]),
        "g_x2": rel(host(out["gx2"]), ref["gx2"]),
        "g_x1": rel(host(out["gx1"]), ref["gx1"]),
    }
    # dL/dtheta = dL/dx1 + sum_g dL/dx3 (F's Jacobian is the identity), as
    # the Adam kernel sums it from the step's buffers
    grad = host(out["gx1"]).sum(axis=0) + host(out["gx3"]).sum(axis=(0, 1))
    errs["grad"] = rel(grad, ref["grad"])
    # Adam divides every element by its own gradient scale, so elements with
    # small gradients carry their relative error into the update: the
    # updated theta is compared with the oracle's (gradient from the oracle),
    # and the update itself with the oracle's Adam on the step's gradient
    theta, m1, v1, step_no = ref["adam"]
    th_o, _, _ = O.adam_step(theta, ref["grad"], m1, v1, step_no, lr=BN.LR)
    th_g, _, _ = O.adam_step(theta, grad, m1, v1, step_no, lr=BN.LR)
    errs["theta"] = rel(host(out["theta"]), th_o)
    errs["dtheta"] = rel(host(out["theta"]) - theta, th_g - theta)
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, f"beyond {tol}: {bad} (all: {errs})"
    return errs


def _eager(arm, idx, g, st):
    _load(arm, idx, g, st)
    arm.step()
    return _outputs(arm)


def _replay(S, arm, idx, g, st):
    """The benchmark's graph: the draws kernel loads the step's row of a
    resident table, then the step; captured once, replayed once."""
    stream = torch.cuda.Stream()
    table = torch.from_numpy(arm.pack_params(idx[None], g[None], st[3])).cuda()
    counter = torch.zeros(1, dtype=torch.int32, device="cuda")
    with torch.cuda.stream(stream):
        _load(arm, idx, g, st)
        arm.step()   # the library's one-time set-up happens outside the capture
        stream.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            S.step_draws(table, counter, arm.params)
            arm.step()
        _load(arm, idx, g, st)
        arm.params.zero_()     # the draws must come from the table
        counter.zero_()
        graph.replay()
        stream.synchronize()
    assert counter.item() == 1
    return _outputs(arm)


@pytest.mark.parametrize("dtype", ["f32", "bf16"])
def test_bench_step_matches_oracle(S, prob, dtype):
    arm, idx, g, st = _arm(S, prob, dtype)
    # the launch form the headline step takes: A's band sums with the MC
    # image riding along (reported by the library, and counted by the bench)
    assert S.ei_fwd_form(arm.plan, 1, 4, arm.idx, arm.idx) == 1
    out = _eager(arm, idx, g, st)
    out["y"] = host(arm.y)
    ref = _oracle(prob, out, idx, g, st)
    _compare(out, ref, TOL[dtype])
    assert arm.plan.status() == 0

    # one replay of the captured step: bitwise the eager step, hence the
    # same parity
    rep = _replay(S, arm, idx, g, st)
    for k in out:
        if isinstance(out[k], torch.Tensor):
            assert torch.equal(out[k], rep[k]), k


def test_bench_step_plain_arm_matches_oracle(S, prob):
    """The plain full-operator arm (all 60 views for both terms) the
    benchmark compares against."""
    plan = S.Plan(BN.N_IMG, BN.N_VIEWS, prob["angs"])
    arm = BN.Arm(S, plan, prob, BN.PLAIN, "f32", torch.device("cuda"))
    idx_all, g_all = BN.step_params(1, BN.PLAIN, first=3)
    st = _state(BN.N_IMG, seed=6)
    out = _eager(arm, idx_all[0], g_all[0], st)
    theta, m1, v1, step_no = (np.asarray(a, dtype=np.float64) if i < 3 else a
                              for i, a in enumerate(st))
    angs, y = prob["angs"], host(arm.y)
    x1 = host(out["x1"])
    r, x2, z = O.ei_stage1(x1, y, angs, None, None, g_all[0])
    x3 = z + theta[None, None]
    loss, mc, ei, gx2, gx3 = O.ei_finish(x2, x3, r, BN.LAM, 1.0)
    gx1 = O.ei_backward(r, gx2, gx3, angs, None, None, g_all[0], 1.0)
    ref = dict(r=r, x2=x2, z=z, x3=x3, loss=loss, mc=mc, ei=ei, gx2=gx2, gx1=gx1,
               grad=gx1.sum(axis=0) + gx3.sum(axis=(0, 1)), y_mc=np.asarray(y),
               adam=(theta, m1, v1, step_no))
    _compare(out, ref, TOL["f32"])
