"""Pins of the oracle's batch-statistics BN layer (Sec. 3.3) and of the
residual CNN stand-in used for BN-only test-time training: closed forms of
the normalised output, the ReLU as a clamp, the backward against central
finite differences and against torch's own batch_norm autograd in float64,
the convolution step against a plain loop, and the residual structure."""
import numpy as np
import pytest

import oracle as O
from paper_2411_05771_gb300 import inputs as I


def _data(shape=(3, 4, 5, 7), seed=0):
    rng = np.random.default_rng(seed)
    v = rng.standard_normal(shape) * 2.0 + 0.7
    C = shape[1]
    scale = 1.0 + 0.3 * rng.standard_normal(C)
    shift = 0.2 * rng.standard_normal(C)
    return rng, v, scale, shift


def test_bn_closed_forms():
    """Without the ReLU each channel of the output has mean = shift and
    variance = scale^2 var / (var + eps) over the batch."""
    _, v, scale, shift = _data()
    eps = 1e-3
    out = O.bn_act(v, scale, shift, relu=False, eps=eps)
    axes = (0, 2, 3)
    var = v.var(axis=axes)
    np.testing.assert_allclose(out.mean(axis=axes), shift, atol=1e-12)
    np.testing.assert_allclose(out.var(axis=axes), scale ** 2 * var / (var + eps), rtol=1e-12)


def test_bn_relu_is_the_clamped_affine_output():
    _, v, scale, shift = _data(seed=1)
    np.testing.assert_array_equal(O.bn_act(v, scale, shift, relu=True),
                                  np.maximum(O.bn_act(v, scale, shift, relu=False), 0.0))


@pytest.mark.parametrize("relu", [False, True])
def test_bn_backward_vs_finite_differences(relu):
    rng, v, scale, shift = _data((2, 3, 4, 5), seed=2)
    g = rng.standard_normal(v.shape)
    f = lambda vv, sc, sh: float(np.sum(g * O.bn_act(vv, sc, sh, relu=relu)))
    g_v, g_scale, g_shift = O.bn_act_bwd(v, g, scale, shift, relu=relu)
    h = 1e-6
    for _ in range(12):
        idx = tuple(int(rng.integers(0, s)) for s in v.shape)
        vp, vm = v.copy(), v.copy()
        vp[idx] += h
        vm[idx] -= h
        fd = (f(vp, scale, shift) - f(vm, scale, shift)) / (2 * h)
        assert abs(fd - g_v[idx]) <= 1e-6 * (1 + abs(fd))
    for c in range(v.shape[1]):
        e = np.zeros_like(scale)
        e[c] = h
        fd_s = (f(v, scale + e, shift) - f(v, scale - e, shift)) / (2 * h)
        fd_b = (f(v, scale, shift + e) - f(v, scale, shift - e)) / (2 * h)
        assert abs(fd_s - g_scale[c]) <= 1e-6 * (1 + abs(fd_s))
        assert abs(fd_b - g_shift[c]) <= 1e-6 * (1 + abs(fd_b))


def test_bn_matches_torch_batch_norm_float64():
    torch = pytest.importorskip("torch")
    rng, v, scale, shift = _data((2, 5, 6, 3), seed=3)
    g = rng.standard_normal(v.shape)
    vt = torch.tensor(v, requires_grad=True)
    st = torch.tensor(scale, requires_grad=True)
    bt = torch.tensor(shift, requires_grad=True)
    out = torch.relu(torch.nn.functional.batch_norm(vt, None, None, st, bt, training=True,
                                                    eps=1e-5))
    out.backward(torch.tensor(g))
    np.testing.assert_allclose(O.bn_act(v, scale, shift), out.detach().numpy(), atol=1e-12)
    g_v, g_s, g_b = O.bn_act_bwd(v, g, scale, shift)
    np.testing.assert_allclose(g_v, vt.grad.numpy(), atol=1e-10)
    np.testing.assert_allclose(g_s, st.grad.numpy(), atol=1e-10)
    np.testing.assert_allclose(g_b, bt.grad.numpy(), atol=1e-10)


def _conv_loop(h, w):
    """3x3 cross-correlation with zero padding 1, written out."""
    n, cin, H, W = h.shape
    cout = w.shape[0]
    out = np.zeros((n, cout, H, W))
    for b in range(n):
        for o in range(cout):
            for i in range(H):
                for j in range(W):
                    s = 0.0
                    for c in range(cin):
                        for di in range(3):
                            for dj in range(3):
                                ii, jj = i + di - 1, j + dj - 1
                                if 0 <= ii < H and 0 <= jj < W:
                                    s += w[o, c, di, dj] * h[b, c, ii, jj]
                    out[b, o, i, j] = s
    return out


def test_rescnn_equals_the_written_out_network():
    wts = I.cnn_weights(channels=3, layers=3, seed=4)
    u = np.random.default_rng(5).standard_normal((2, 6, 5))
    h = u[:, None]
    C = wts.channels
    for l, w in enumerate(wts.conv):
        h = _conv_loop(h, w)
        if l < wts.layers - 1:
            o = 2 * C * l
            h = O.bn_act(h, wts.bn[o:o + C], wts.bn[o + C:o + 2 * C])
    np.testing.assert_allclose(O.rescnn(u, wts.conv, wts.bn), u + h[:, 0], atol=1e-12)


def test_rescnn_is_the_identity_without_its_last_layer():
    wts = I.cnn_weights(channels=4, layers=3, seed=6)
    conv = list(wts.conv)
    conv[-1] = np.zeros_like(conv[-1])
    u = np.random.default_rng(7).standard_normal((3, 8, 8))
    np.testing.assert_array_equal(O.rescnn(u, conv, wts.bn), u)


def test_ttt_bn_loss_with_identity_network_is_the_plain_loss():
    """With the residual branch off, the BN-only loss is the residual-network
    loss at theta = 0."""
    N, n_ang, G = 12, 8, 2
    wts = I.cnn_weights(channels=2, layers=2, seed=8)
    conv = [w for w in wts.conv]
    conv[-1] = np.zeros_like(conv[-1])
    rng = np.random.default_rng(9)
    x0 = rng.standard_normal((1, N, N))
    ang = I.uniform_angles(n_ang)
    y = rng.standard_normal((1, n_ang, O.ndet(N)))
    g = rng.uniform(0, 360, size=(1, G))
    idx = I.sketch_indices(n_ang, 4, 1)
    a = O.ttt_bn_loss(wts.bn, conv, x0, y, ang, None, idx, g, 0.7, 1.0)
    b = O.ttt_loss(np.zeros((N, N)), x0, y, ang, None, idx, g, 0.7, 1.0)[0]
    assert abs(a - b) <= 1e-12 * abs(b)
