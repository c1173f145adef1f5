"""GPU parity of the multi-coil MRI path (Sec. 3.4, Eq. (e:mri), Algorithm 3)
against the FP64 oracle: A, A^H, A^dagger with and without mask, residual
and image weight, on power-of-two sizes 8 .. 128 and 1 .. 15 coils; the
adjoint identity; dinv; coil mixing; rotations of two-channel images; the
PCA coil compression and coil sketch; and the coil-sketched EI step's loss
and gradient."""
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


def dev(a):
    return torch.tensor(np.asarray(a), dtype=torch.float32, device="cuda")


def host(t):
    return t.detach().double().cpu().numpy()


@pytest.mark.parametrize("N,Nc,B", [(8, 1, 1), (16, 3, 2), (32, 15, 1), (64, 4, 3),
                                    (128, 15, 1), (256, 2, 1)])
@pytest.mark.parametrize("masked", [False, True])
def test_mri_operators_match_oracle(S, N, Nc, B, masked):
    rng = np.random.default_rng(N + Nc)
    maps = I.coil_maps(Nc, N, seed=N)
    mask = I.undersampling_mask(N, seed=N) if masked else None
    x = np.stack([I.complex_phantom(b, N) for b in range(B)])
    k = rng.standard_normal((B, Nc, 2, N, N))
    aux = rng.standard_normal((B, Nc, 2, N, N))
    xw = rng.uniform(0.5, 2.0, (N, N))
    md = None if mask is None else dev(mask)
    ref_k = O.mri_fwd(x, maps, mask)
    assert rel(host(S.mri_fwd(dev(x), dev(maps), md)), ref_k) <= FP32_TOL
    got = S.mri_fwd(dev(x), dev(maps), md, aux=dev(aux), alpha=0.5)
    assert rel(host(got), 0.5 * (aux - ref_k)) <= FP32_TOL
    got = S.mri_fwd(dev(x), dev(maps), md, xw=dev(xw))
    assert rel(host(got), O.mri_fwd(x * xw, maps, mask)) <= FP32_TOL
    ref_x = O.mri_adj(k, maps, mask)
    assert rel(host(S.mri_adj(dev(k), dev(maps), md)), ref_x) <= FP32_TOL
    dinv = S.mri_dinv(dev(maps))
    assert rel(host(dinv), O.mri_dinv(maps)) <= FP32_TOL
    out = dev(x)
    S.mri_adj(dev(k), dev(maps), md, dinv, alpha=2.0, beta=-1.0, out=out)
    assert rel(host(out), 2.0 * O.mri_pinv(k, maps, mask) - x) <= FP32_TOL


def test_mri_adjoint_identity_on_gpu(S):
    N, Nc = 128, 8
    rng = np.random.default_rng(3)
    maps, mask = dev(I.coil_maps(Nc, N)), dev(I.undersampling_mask(N))
    x = dev(rng.standard_normal((2, 2, N, N)))
    k = dev(rng.standard_normal((2, Nc, 2, N, N)))
    lhs = float((S.mri_fwd(x, maps, mask).double() * k.double()).sum())
    rhs = float((x.double() * S.mri_adj(k, maps, mask).double()).sum())
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


def test_mri_rejects_bad_sizes(S):
    maps = torch.zeros((2, 2, 24, 24), device="cuda")
    with pytest.raises(RuntimeError):
        S.mri_fwd(torch.zeros((1, 2, 24, 24), device="cuda"), maps)


def test_coil_mix_and_two_channel_rotation(S):
    rng = np.random.default_rng(4)
    W = rng.standard_normal((3, 5)) + 1j * rng.standard_normal((3, 5))
    x = rng.standard_normal((2, 5, 2, 16, 16))
    got = S.coil_mix(torch.tensor(W, dtype=torch.complex64, device="cuda"), dev(x))
    assert rel(host(got), O.coil_mix(W, x)) <= FP32_TOL
    img = dev(rng.standard_normal((2, 2, 32, 32)))
    g = torch.tensor(rng.uniform(0, 360, (2, 3)), dtype=torch.float64, device="cuda")
    both = S.rotate(img, g)                                        # [2, 3, 2, 32, 32]
    for c in range(2):
        assert torch.equal(both[:, :, c], S.rotate(img[:, c].contiguous(), g))
    gout = dev(rng.standard_normal((2, 3, 2, 32, 32)))
    adj = S.rotate_adj(gout, g)
    for c in range(2):
        assert torch.equal(adj[:, c], S.rotate_adj(gout[:, :, c].contiguous(), g))


def _mri_problem(N=32, Nc=8, seed=0):
    rng = np.random.default_rng(seed)
    maps = I.coil_maps(Nc, N, seed=seed)
    mask = I.undersampling_mask(N, seed=seed)
    x_gt = I.complex_phantom(seed, N)[None]
    y = O.mri_fwd(x_gt, maps, mask) + 0.01 * rng.standard_normal((1, Nc, 2, N, N)) * mask
    return maps, mask, y


def test_coil_sketch_matches_oracle(S):
    from paper_2411_05771_gb300.mri import CoilSketch
    maps, mask, y = _mri_problem()
    L, R = 6, 2
    s_low = I.rademacher(np.random.default_rng(5), (2, L - R))
    y_d = dev(y)
    cs = CoilSketch(y_d, dev(maps), L, R, s_low)
    # the oracle on the same FP32-stored k-space (the covariance and its
    # eigenvectors are FP64 on both sides)
    y32 = host(y_d)
    Q, _ = O.coil_pca(y32[0], L)
    assert np.abs(cs.Q.cpu().numpy() - Q).max() <= 1e-9
    W = O.coil_sketch(L, R, s_low) @ Q.T
    assert rel(host(cs.maps), O.coil_mix(W, maps[None])[0]) <= FP32_TOL
    assert rel(host(cs.y), O.coil_mix(W, y32)) <= FP32_TOL


@pytest.mark.parametrize("sketch", [False, True])
def test_csk_step_loss_and_gradient_match_oracle(S, sketch):
    from paper_2411_05771_gb300.mri import CoilSketch, CskArm
    maps, mask, y = _mri_problem(seed=1)
    N, G = 32, 2
    rng = np.random.default_rng(6)
    x0 = O.mri_pinv(y, maps, mask)
    if sketch:
        L, R = 6, 1
        s_low = I.rademacher(np.random.default_rng(7), (1, L - R))
        cs = CoilSketch(dev(y), dev(maps), L, R, s_low)
        m_d, y_d, dinv_d = cs.maps, cs.y, cs.dinv
        y32 = host(dev(y))
        W = O.coil_sketch(L, R, s_low) @ O.coil_pca(y32[0], L)[0].T
        m_o, y_o = O.coil_mix(W, maps[None])[0], O.coil_mix(W, y32)
    else:
        m_d, y_d = dev(maps), dev(y)
        dinv_d = S.mri_dinv(m_d)
        m_o, y_o = maps, y
    arm = CskArm(dev(x0), y_d, m_d, dev(mask), dinv_d, G, lam=0.7)
    theta = 0.05 * rng.standard_normal((2, N, N))
    g = rng.uniform(0, 360, (1, G))
    arm.theta.copy_(dev(theta))
    arm.g.copy_(torch.tensor(g))
    arm.grad()
    loss_o, grad_o, _ = O.mri_ttt_grad(theta, x0, y_o, m_o, mask, g, 0.7)
    assert abs(arm.loss.item() - loss_o) <= 1e-4 * abs(loss_o)
    grad = host(arm.gx1)[0] + host(arm.gx3)[0].sum(axis=0)
    assert rel(grad, grad_o) <= 1e-4
