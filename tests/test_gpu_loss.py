"""GPU parity of the fused EI / SkEI loss (Eq. e:skeiloss; Algorithm 2) and
its hand-written backward against the FP64 oracle, plus central finite
differences through the autograd wrappers.

Workload of the differentiated step: batch 8 x G=4 rotations, 256^2, MC on
all 180 angles, EI on a 45-angle sketch (stride 4, random offset)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2411_05771_gb300 import inputs as I

pytestmark = pytest.mark.gpu
FP32_TOL = 1e-5


@pytest.fixture(scope="module")
def S():
    from paper_2411_05771_gb300 import skei
    return skei


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def dev(a, dtype=torch.float32):
    return torch.tensor(np.asarray(a), dtype=dtype, device="cuda")


def host(t):
    return t.detach().double().cpu().numpy()


def _setup(N, n_ang, B, G, m, sketch_mc, seed=0):
    rng = np.random.default_rng(seed)
    x_gt = np.stack([I.rasterize(I.random_ellipses(seed + b), N) for b in range(B)])
    angs = I.uniform_angles(n_ang)
    nd = O.ndet(N)
    y = O.proj_fwd(x_gt, angs, nd) + 0.5 * rng.standard_normal((B, n_ang, nd))
    x1 = x_gt + 0.05 * rng.standard_normal((B, N, N))
    step = I.step_rng(seed)
    off = I.random_sketch_offset(step, n_ang, m)
    idx = I.sketch_indices(n_ang, m, off)
    g = I.rotation_angles(step, B, G)
    mc_idx = idx if sketch_mc else None
    return dict(angs=angs, nd=nd, y=y, x1=x1, idx=idx, g=g, mc_idx=mc_idx)


@pytest.mark.parametrize("N,n_ang,B,G,m,sketch_mc", [
    (256, 180, 8, 4, 45, False),   # the differentiated 256^2 step
    (64, 60, 2, 3, 15, True),      # sketched MC as in Algorithm 2
    (37, 24, 3, 2, 6, True),       # ragged sizes
    (64, 60, 2, 4, 15, True),      # G = 4, shared sketch: MC images ride with EI groups
    (100, 30, 1, 4, 10, True),     # the same, one ragged image
    (256, 180, 8, 4, 45, True),    # riding MC images at 256^2 (the shared-memory opt-in)
])
def test_ei_step_matches_oracle(S, N, n_ang, B, G, m, sketch_mc):
    P = _setup(N, n_ang, B, G, m, sketch_mc)
    plan = S.Plan(N, n_ang)
    lam = 0.7
    mc_scale = n_ang / m if sketch_mc else 1.0
    idx_d = dev(P["idx"], torch.int32)
    mc_d = idx_d if sketch_mc else None
    g_d = dev(P["g"], torch.float64)
    x1 = dev(P["x1"])
    # x3 = F(z) with F(u) = u + theta
    theta = 0.01 * np.random.default_rng(1).standard_normal((N, N))
    r, x2, z = S.ei_loss_fwd(plan, x1, dev(P["y"]), g_d, mc_idx=mc_d, sk_idx=idx_d)
    x3 = S.residual_add(z, dev(theta))
    loss, mc, ei, g_x2, g_x3 = S.ei_loss_finish(x2, x3, r, lam, mc_scale)
    g_x1 = S.ei_loss_bwd(plan, r, g_x2, g_x3, g_d, mc_scale / B, mc_idx=mc_d, sk_idx=idx_d)

    x1_64 = host(x1)
    r_o, x2_o, z_o = O.ei_stage1(x1_64, P["y"], P["angs"], P["mc_idx"], P["idx"], P["g"])
    x3_o = z_o + theta[None, None]
    loss_o, mc_o, ei_o, gx2_o, gx3_o = O.ei_finish(x2_o, x3_o, r_o, lam, mc_scale)
    gx1_o = O.ei_backward(r_o, gx2_o, gx3_o, P["angs"], P["mc_idx"], P["idx"], P["g"], mc_scale)
    y_mc = P["y"] if P["mc_idx"] is None else P["y"][:, P["mc_idx"]]
    # the residual's FP32 error is bounded relative to its operands
    assert np.linalg.norm(host(r) - r_o) <= FP32_TOL * np.linalg.norm(y_mc)
    assert rel(host(x2), x2_o) <= FP32_TOL
    assert rel(host(z), z_o) <= FP32_TOL
    assert rel(host(g_x2), gx2_o) <= FP32_TOL
    assert rel(host(g_x3), gx3_o) <= FP32_TOL
    assert rel(host(g_x1), gx1_o) <= FP32_TOL
    assert abs(loss.item() - loss_o) <= FP32_TOL * abs(loss_o)
    assert rel(host(mc), mc_o) <= FP32_TOL
    assert rel(host(ei), ei_o) <= FP32_TOL


def test_full_sketch_equals_plain(S):
    N, n_ang, B, G = 48, 24, 2, 2
    P = _setup(N, n_ang, B, G, 24, False)
    plan = S.Plan(N, n_ang)
    g_d = dev(P["g"], torch.float64)
    all_idx = torch.arange(n_ang, dtype=torch.int32, device="cuda")
    a = S.ei_loss_fwd(plan, dev(P["x1"]), dev(P["y"]), g_d)
    b = S.ei_loss_fwd(plan, dev(P["x1"]), dev(P["y"]), g_d, mc_idx=all_idx, sk_idx=all_idx)
    for u, v in zip(a, b):
        assert torch.equal(u, v)


def test_autograd_gradient_vs_oracle_and_finite_differences(S):
    """F(u) = u + theta; d loss / d theta through the autograd wrappers
    against the oracle's analytic gradient and against central differences
    (h = 1e-3) of the GPU loss at 64 random pixels."""
    from paper_2411_05771_gb300.autograd import skei_loss
    N, n_ang, B, G, m = 256, 180, 8, 4, 45
    P = _setup(N, n_ang, B, G, m, False, seed=3)
    plan = S.Plan(N, n_ang)
    lam = 1.0
    idx_d = dev(P["idx"], torch.int32)
    g_d = dev(P["g"], torch.float64)
    y_d = dev(P["y"])
    x0 = dev(P["x1"])
    theta = torch.zeros((N, N), device="cuda", requires_grad=True)

    def loss_of(th):
        x1 = x0 + th
        return skei_loss(plan, x1, y_d, lambda z: z + th, g_d, None, idx_d, lam, 1.0)

    L = loss_of(theta)
    L.backward()
    g = host(theta.grad)
    L_o, g_o, _ = O.ttt_grad(np.zeros((N, N)), host(x0), P["y"], P["angs"], None, P["idx"],
                             P["g"], lam, 1.0)
    assert abs(L.item() - L_o) <= FP32_TOL * abs(L_o)
    assert rel(g, g_o) <= 1e-4
    rng = np.random.default_rng(11)
    h = 1e-3
    pix = rng.choice(N * N, 64, replace=False)
    fd = []
    with torch.no_grad():
        for q in pix:
            e = torch.zeros(N * N, device="cuda")
            e[q] = h
            e = e.reshape(N, N)
            fd.append((loss_of(e).item() - loss_of(-e).item()) / (2 * h))
    fd = np.array(fd)
    an = g.ravel()[pix]
    assert np.abs(fd - an).max() <= 1e-3 * np.abs(g).max() + 2e-3 * np.abs(an).max()


# ------------------------------------------------- a sketch per measurement
@pytest.mark.parametrize("N,n_ang,B,G,m,sketch_mc", [
    (256, 180, 8, 4, 45, False),   # Algorithm 1 over 8 measurements, MC on all views
    (64, 60, 3, 4, 15, True),      # sketched MC: each MC image rides with its EI group
    (37, 24, 3, 3, 6, True),       # G = 3: groups of 4 would straddle samples
    (100, 30, 5, 2, 10, False),    # G = 2, ragged
])
def test_per_sample_sketches_match_oracle(S, N, n_ang, B, G, m, sketch_mc):
    P = _setup(N, n_ang, B, G, m, sketch_mc, seed=N + B)
    rng = np.random.default_rng(N * B)
    rows = np.stack([I.sketch_indices(n_ang, m, int(rng.integers(0, n_ang // m)))
                     for _ in range(B)]).astype(np.int32)
    plan = S.Plan(N, n_ang)
    lam = 0.7
    mc_scale = n_ang / m if sketch_mc else 1.0
    rows_d = dev(rows, torch.int32)
    mc_d = rows_d if sketch_mc else None
    mc_rows = rows if sketch_mc else None
    g_d = dev(P["g"], torch.float64)
    x1 = dev(P["x1"])
    theta = 0.01 * np.random.default_rng(2).standard_normal((N, N))
    r, x2, z = S.ei_loss_fwd_per_sample(plan, x1, dev(P["y"]), g_d, mc_idx=mc_d, sk_idx=rows_d)
    x3 = S.residual_add(z, dev(theta))
    loss, mc, ei, g_x2, g_x3 = S.ei_loss_finish(x2, x3, r, lam, mc_scale)
    g_x1 = S.ei_loss_bwd_per_sample(plan, r, g_x2, g_x3, g_d, mc_scale / B, mc_idx=mc_d,
                                    sk_idx=rows_d)

    r_o, x2_o, z_o = O.ei_stage1_per_sample(host(x1), P["y"], P["angs"], mc_rows, rows, P["g"])
    x3_o = z_o + theta[None, None]
    loss_o, mc_o, ei_o, gx2_o, gx3_o = O.ei_finish(x2_o, x3_o, r_o, lam, mc_scale)
    gx1_o = O.ei_backward_per_sample(r_o, gx2_o, gx3_o, P["angs"], mc_rows, rows, P["g"],
                                     mc_scale)
    y_mc = (P["y"] if mc_rows is None
            else np.stack([P["y"][b][rows[b]] for b in range(B)]))
    assert np.linalg.norm(host(r) - r_o) <= FP32_TOL * np.linalg.norm(y_mc)
    assert rel(host(z), z_o) <= FP32_TOL
    assert rel(host(g_x1), gx1_o) <= FP32_TOL
    assert abs(loss.item() - loss_o) <= FP32_TOL * abs(loss_o)
    assert rel(host(ei), ei_o) <= FP32_TOL


@pytest.mark.parametrize("sketch_mc", [False, True])
def test_per_sample_with_equal_rows_is_the_shared_sketch_bitwise(S, sketch_mc):
    """The same sketch in every row runs the same kernels in the same order
    as the shared-sketch entry points: identical bits."""
    N, n_ang, B, G, m = 64, 60, 3, 4, 15
    P = _setup(N, n_ang, B, G, m, sketch_mc, seed=9)
    plan = S.Plan(N, n_ang)
    idx_d = dev(P["idx"], torch.int32)
    rows_d = idx_d.repeat(B, 1).contiguous()
    g_d = dev(P["g"], torch.float64)
    x1, y = dev(P["x1"]), dev(P["y"])
    a = S.ei_loss_fwd(plan, x1, y, g_d, mc_idx=idx_d if sketch_mc else None, sk_idx=idx_d)
    b = S.ei_loss_fwd_per_sample(plan, x1, y, g_d, mc_idx=rows_d if sketch_mc else None,
                                 sk_idx=rows_d)
    for u, v in zip(a, b):
        assert torch.equal(u, v)
    r, x2, z = a
    gx = 0.1 * x2
    ga = S.ei_loss_bwd(plan, r, gx, z, g_d, 0.3, mc_idx=idx_d if sketch_mc else None,
                       sk_idx=idx_d)
    gb = S.ei_loss_bwd_per_sample(plan, r, gx, z, g_d, 0.3,
                                  mc_idx=rows_d if sketch_mc else None, sk_idx=rows_d)
    assert torch.equal(ga, gb)


def test_forward_form_query(S):
    """skei_ei_fwd_form: the riding band-sums form where the MC and EI terms
    share one list with G = 4; the cluster form for a small launch
    otherwise; bad sizes are refused."""
    plan = S.Plan(64, 60)
    idx = dev(I.sketch_indices(60, 15, 1), torch.int32)
    other = idx.clone()
    assert S.ei_fwd_form(plan, 2, 4, idx, idx) == 1
    assert S.ei_fwd_form(plan, 2, 4, other, idx) == 0
    assert S.ei_fwd_form(plan, 2, 3, idx, idx) == 0
    rows = idx.repeat(2, 1).contiguous()
    assert S.ei_fwd_form(plan, 2, 4, rows, rows, per_sample=True) == 1
    with pytest.raises(RuntimeError):
        S.ei_fwd_form(plan, 0, 4, idx, idx)
