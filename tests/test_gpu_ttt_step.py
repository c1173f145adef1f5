"""skei_ttt_residual_step: Algorithm 2's iteration for the network
F_theta(u) = u + theta in one call, with the network and Adam folded into
the operator launches.  Every result must be bitwise that of the separate
calls (skei_residual_add, skei_ei_loss_fwd / finish / bwd, skei_adam_step),
whose parity with the FP64 oracle the other tests establish (the 512^2
benchmark step: tests/test_gpu_bench_step.py)."""
import numpy as np
import pytest
import torch

from paper_2411_05771_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from paper_2411_05771_gb300 import skei
    return skei


def _separate(S, plan, x0, theta, m, v, step, y, g, mc_idx, sk_idx, lam, mc_scale, lr):
    B = x0.shape[0]
    x1 = S.residual_add(x0, theta)
    r, x2, z = S.ei_loss_fwd(plan, x1, y, g, mc_idx, sk_idx)
    x3 = S.residual_add(z, theta)
    loss, mc, ei, gx2, gx3 = S.ei_loss_finish(x2, x3, r, lam, mc_scale)
    gx1 = S.ei_loss_bwd(plan, r, gx2, gx3, g, mc_scale / B, mc_idx, sk_idx)
    S.adam_step(theta, m, v, step, gx1, gx3, lr=lr)
    return dict(x1=x1, r=r, x2=x2, z=z, x3=x3, gx2=gx2, gx3=gx3, gx1=gx1, loss=loss, mc=mc,
                ei=ei, theta=theta, m=m, v=v)


@pytest.mark.parametrize("N,n_ang,B,G,m,sketch_mc,dtype", [
    (512, 60, 1, 4, 30, True, torch.float32),     # the benchmark's step
    (512, 60, 1, 4, 30, True, torch.bfloat16),
    (512, 60, 1, 4, 60, False, torch.float32),    # the plain arm: all angles
    (64, 60, 2, 4, 15, True, torch.float32),      # two measurements: Adam on its own
    (37, 24, 1, 3, 6, True, torch.float32),       # ragged, G = 3
    # 8 measurements at 256^2 with the MC images riding in A's band sums:
    # 46 KB of dynamic shared memory, under the 48 KB default on its own but
    # not with the kernel's static part (the launch must opt in)
    (256, 180, 8, 4, 45, True, torch.float32),
    (256, 180, 8, 4, 180, False, torch.float32),  # the plain form: all angles, both terms
    (100, 36, 2, 4, 12, True, torch.bfloat16),    # N % 8 = 4, BF16 storage, riding MC images
])
def test_fused_step_is_bitwise_the_separate_calls(S, N, n_ang, B, G, m, sketch_mc, dtype):
    rng = np.random.default_rng(N + m)
    plan = S.Plan(N, n_ang)
    dev = "cuda"
    x0 = torch.tensor(np.stack([I.rasterize(I.random_ellipses(b), N) for b in range(B)]),
                      device=dev).to(dtype)
    y = torch.tensor(rng.standard_normal((B, n_ang, plan.n_det)), device=dev).to(dtype)
    g = torch.tensor(I.rotation_angles(rng, B, G), dtype=torch.float64, device=dev)
    idx = None if m == n_ang else torch.tensor(
        I.sketch_indices(n_ang, m, I.random_sketch_offset(rng, n_ang, m)), dtype=torch.int32,
        device=dev)
    mc_idx = idx if sketch_mc else None
    mc_scale = n_ang / m if sketch_mc else 1.0
    lam, lr = 0.7, 5e-4
    f32 = dict(dtype=torch.float32, device=dev)
    theta0 = torch.tensor(0.01 * rng.standard_normal((N, N)), **f32)
    m0 = torch.tensor(1e-4 * rng.standard_normal((N, N)), **f32)
    v0 = torch.tensor((1e-4 * rng.standard_normal((N, N))) ** 2, **f32)
    step = torch.full((), 5, dtype=torch.int32, device=dev)

    ref = _separate(S, plan, x0, theta0.clone(), m0.clone(), v0.clone(), step, y, g, mc_idx, idx,
                    lam, mc_scale, lr)
    th, mm, vv = theta0.clone(), m0.clone(), v0.clone()
    out = S.ttt_residual_step(plan, x0, th, mm, vv, step, y, g, mc_idx, idx, lam, mc_scale, lr)
    torch.cuda.synchronize()
    got = dict(zip(("x1", "r", "x2", "z", "x3", "gx2", "gx3", "gx1", "loss", "mc", "ei"), out))
    got.update(theta=th, m=mm, v=vv)
    for k in ref:
        assert torch.equal(got[k], ref[k]), k
    assert plan.status() == 0


def test_fused_step_in_a_graph_replays_bitwise(S):
    """Captured once, the fused step replays to the eager results."""
    N, n_ang, G, m = 64, 60, 4, 15
    rng = np.random.default_rng(3)
    plan = S.Plan(N, n_ang)
    x0 = torch.tensor(I.rasterize(I.random_ellipses(1), N)[None], device="cuda",
                      dtype=torch.float32)
    y = torch.randn(1, n_ang, plan.n_det, device="cuda")
    g = torch.tensor(I.rotation_angles(rng, 1, G), dtype=torch.float64, device="cuda")
    idx = torch.tensor(I.sketch_indices(n_ang, m, 2), dtype=torch.int32, device="cuda")
    step = torch.ones((), dtype=torch.int32, device="cuda")
    state = [torch.zeros(N, N, device="cuda") for _ in range(3)]
    work = torch.empty(S.ttt_residual_workspace_size(plan, S.F32, 1, G, m, m), dtype=torch.uint8,
                       device="cuda")
    out = S.ttt_residual_step(plan, x0, *state, step, y, g, idx, idx, 1.0, n_ang / m, work=work)
    eager = [t.clone() for t in out] + [t.clone() for t in state]
    for t in state:
        t.zero_()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=stream):
            S.ttt_residual_step(plan, x0, *state, step, y, g, idx, idx, 1.0, n_ang / m,
                                out=out, work=work)
        for t in state:
            t.zero_()
        graph.replay()
        stream.synchronize()
    for a, b in zip(eager, list(out) + state):
        assert torch.equal(a, b)
