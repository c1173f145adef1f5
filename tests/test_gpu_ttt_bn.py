"""GPU parity of BN-only test-time training (Sec. 3.3): the batch-statistics
BN kernels (skei_bn_act_fwd / skei_bn_act_bwd) against the FP64 oracle on
ragged shapes and both storage types, and the whole TTT-BN-SkEI step (CNN
stand-in + operators + loss) against the oracle's loss and its central
finite-difference gradient in the BN parameters; the step replays from a
CUDA graph with the eager step's bits."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2411_05771_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5
BF16_TOL = 1e-2


@pytest.fixture(scope="module", autouse=True)
def strict_fp32():
    """FP32 convolutions without TF32 and deterministic cuDNN algorithms, so
    that the network around the kernels is a plain FP32 computation."""
    saved = (torch.backends.cudnn.allow_tf32, torch.backends.cuda.matmul.allow_tf32,
             torch.backends.cudnn.deterministic, torch.backends.cudnn.benchmark)
    torch.backends.cudnn.allow_tf32 = False
    torch.backends.cuda.matmul.allow_tf32 = False
    torch.backends.cudnn.deterministic = True
    torch.backends.cudnn.benchmark = False
    yield
    (torch.backends.cudnn.allow_tf32, torch.backends.cuda.matmul.allow_tf32,
     torch.backends.cudnn.deterministic, torch.backends.cudnn.benchmark) = saved


@pytest.fixture(scope="module")
def S():
    from paper_2411_05771_gb300 import skei
    return skei


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def host(t):
    return t.detach().double().cpu().numpy()


# (B, C, H, W): one chunk and several, ragged tails, HW not a multiple of 4,
# one channel, many channels
SHAPES = [(1, 1, 5, 7), (2, 3, 16, 16), (4, 16, 64, 64), (1, 32, 70, 70), (3, 5, 100, 129),
          (2, 2, 181, 181)]


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("relu", [True, False])
def test_bn_act_forward_backward_vs_oracle(S, shape, relu):
    gen = torch.Generator().manual_seed(sum(shape))
    C = shape[1]
    v = (torch.randn(shape, generator=gen) * 2.0 + 0.7).cuda()
    scale = (1.0 + 0.3 * torch.randn(C, generator=gen)).cuda()
    shift = (0.2 * torch.randn(C, generator=gen)).cuda()
    g = torch.randn(shape, generator=gen).cuda()
    out, mean, rstd = S.bn_act_fwd(v, scale, shift, relu)
    ref = O.bn_act(host(v), host(scale), host(shift), relu)
    assert rel(host(out), ref) <= FP32_TOL
    vv = host(v)
    axes = (0, 2, 3)
    np.testing.assert_allclose(host(mean), vv.mean(axis=axes), rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(host(rstd), 1.0 / np.sqrt(vv.var(axis=axes) + 1e-5), rtol=1e-5)
    g_v, g_s, g_b = S.bn_act_bwd(v, g, scale, shift, mean, rstd, relu)
    rg_v, rg_s, rg_b = O.bn_act_bwd(vv, host(g), host(scale), host(shift), relu)
    assert rel(host(g_v), rg_v) <= FP32_TOL
    assert rel(host(g_s), rg_s) <= FP32_TOL
    assert rel(host(g_b), rg_b) <= FP32_TOL


def test_bn_act_bf16_storage(S):
    gen = torch.Generator().manual_seed(11)
    v = (torch.randn((2, 4, 33, 40), generator=gen) + 0.5).to(torch.bfloat16).cuda()
    scale = (1.0 + 0.3 * torch.randn(4, generator=gen)).cuda()
    shift = (0.2 * torch.randn(4, generator=gen)).cuda()
    g = torch.randn((2, 4, 33, 40), generator=gen).to(torch.bfloat16).cuda()
    out, mean, rstd = S.bn_act_fwd(v, scale, shift)
    assert out.dtype == torch.bfloat16
    assert rel(host(out), O.bn_act(host(v), host(scale), host(shift))) <= BF16_TOL
    g_v, g_s, g_b = S.bn_act_bwd(v, g, scale, shift, mean, rstd)
    rg_v, rg_s, rg_b = O.bn_act_bwd(host(v), host(g), host(scale), host(shift))
    assert rel(host(g_v), rg_v) <= BF16_TOL
    assert rel(host(g_s), rg_s) <= BF16_TOL
    assert rel(host(g_b), rg_b) <= BF16_TOL


def test_bn_act_is_deterministic_and_rejects_bad_input(S):
    gen = torch.Generator().manual_seed(12)
    v = torch.randn((3, 6, 50, 50), generator=gen).cuda()
    scale, shift = torch.ones(6, device="cuda"), torch.zeros(6, device="cuda")
    a = S.bn_act_fwd(v, scale, shift)[0]
    b = S.bn_act_fwd(v, scale, shift)[0]
    assert torch.equal(a, b)
    with pytest.raises(ValueError):
        S.bn_act_fwd(v, scale[:5].contiguous(), shift)
    with pytest.raises(RuntimeError):
        S.bn_act_fwd(v, scale, shift, eps=0.0)


def _ttt_problem(N=16, n_ang=12, B=1, G=2, m=4, C=4, layers=3, seed=0):
    rng = np.random.default_rng(seed)
    wts = I.cnn_weights(channels=C, layers=layers, seed=seed)
    ang = I.uniform_angles(n_ang)
    x_gt = np.stack([I.rasterize(I.random_ellipses(seed + b), N) for b in range(B)])
    y = O.proj_fwd(x_gt, ang, O.ndet(N)) + 0.05 * rng.standard_normal((B, n_ang, O.ndet(N)))
    x0 = O.fbp(y, ang, N)
    g = rng.uniform(0.0, 360.0, size=(B, G))
    idx = I.sketch_indices(n_ang, m, int(rng.integers(0, n_ang // m)))
    return wts, ang, x0, y, g, idx


@pytest.mark.parametrize("B", [1, 2])
def test_ttt_bn_loss_and_gradient_vs_oracle(S, B):
    from paper_2411_05771_gb300.autograd import skei_loss
    from paper_2411_05771_gb300.net import ResCNN
    wts, ang, x0, y, g, idx = _ttt_problem(B=B, seed=B)
    lam, mc_scale = 0.8, 1.0
    plan = S.Plan(x0.shape[-1], len(ang), ang)
    net = ResCNN(wts)
    f32 = dict(dtype=torch.float32, device="cuda")
    x0_d, y_d = torch.tensor(x0, **f32), torch.tensor(y, **f32)
    g_d = torch.tensor(g, dtype=torch.float64, device="cuda")
    idx_d = torch.tensor(idx, dtype=torch.int32, device="cuda")
    loss = skei_loss(plan, net(x0_d), y_d, net, g_d, None, idx_d, lam, mc_scale)
    (grad,) = torch.autograd.grad(loss, [net.bn])
    ref = O.ttt_bn_loss(wts.bn, wts.conv, x0, y, ang, None, idx, g, lam, mc_scale)
    assert abs(float(loss.detach()) - ref) <= 1e-4 * abs(ref)
    h = 1e-5
    fd = np.zeros_like(wts.bn)
    for i in range(wts.bn.size):
        e = np.zeros_like(wts.bn)
        e[i] = h
        fd[i] = (O.ttt_bn_loss(wts.bn + e, wts.conv, x0, y, ang, None, idx, g, lam, mc_scale)
                 - O.ttt_bn_loss(wts.bn - e, wts.conv, x0, y, ang, None, idx, g, lam,
                                 mc_scale)) / (2 * h)
    assert rel(host(grad), fd) <= 1e-3


def test_ttt_bn_step_replays_from_a_cuda_graph(S):
    """Network, operators, loss, autograd backward and Adam on the BN
    parameters, captured as one CUDA graph: a replay gives the eager step's
    parameters bit for bit."""
    from paper_2411_05771_gb300.autograd import skei_loss
    from paper_2411_05771_gb300.net import ResCNN
    wts, ang, x0, y, g, idx = _ttt_problem(N=32, n_ang=16, B=1, G=4, m=8, C=8, seed=3)
    plan = S.Plan(32, 16, ang)
    f32 = dict(dtype=torch.float32, device="cuda")
    x0_d, y_d = torch.tensor(x0, **f32), torch.tensor(y, **f32)
    g_d = torch.tensor(g, dtype=torch.float64, device="cuda")
    idx_d = torch.tensor(idx, dtype=torch.int32, device="cuda")
    step_no = torch.ones((), dtype=torch.int32, device="cuda")

    def make():
        net = ResCNN(wts)
        m1 = torch.zeros_like(net.bn)
        v1 = torch.zeros_like(net.bn)
        return net, m1, v1

    def step(net, m1, v1):
        loss = skei_loss(plan, net(x0_d), y_d, net, g_d, None, idx_d, 1.0, 1.0)
        (gr,) = torch.autograd.grad(loss, [net.bn])
        with torch.no_grad():
            S.adam_step(net.bn.data, m1, v1, step_no, gr, lr=5e-4)
        return loss

    net_e, m_e, v_e = make()
    step(net_e, m_e, v_e)
    torch.cuda.synchronize()

    net_g, m_g, v_g = make()
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    bn0 = net_g.bn.detach().clone()
    with torch.cuda.stream(st):
        for _ in range(2):   # warm-up outside the capture
            step(net_g, m_g, v_g)
    st.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=st):
        step(net_g, m_g, v_g)
    with torch.no_grad():
        net_g.bn.copy_(bn0)
    m_g.zero_()
    v_g.zero_()
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(net_g.bn, net_e.bn)
    assert torch.equal(m_g, m_e) and torch.equal(v_g, v_e)
