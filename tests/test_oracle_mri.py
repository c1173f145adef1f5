"""Pins of the oracle's multi-coil MRI operators and coil sketch (Sec. 3.4,
Eq. (e:mri), Algorithm 3): the DFT's sign and unitary scale against a
written-out sum, the adjoint identity, A^dagger A = I with every sample
taken, Parseval for a unit-modulus coil, the closed form of dinv, coil
mixing against a loop, PCA on data of known rank, the sketch's block
structure, and the C-SkEI gradient against central differences (exact: the
loss is quadratic in theta for F(u) = u + theta)."""
import numpy as np

import oracle as O
from paper_2411_05771_gb300 import inputs as I


def test_dft_convention_is_the_unitary_sum():
    N = 8
    rng = np.random.default_rng(0)
    x = rng.standard_normal((1, 2, N, N))
    one = np.zeros((1, 2, N, N))
    one[0, 0] = 1.0
    k = O.mri_fwd(x, one)[0, 0]
    z = x[0, 0] + 1j * x[0, 1]
    ref = np.zeros((N, N), dtype=complex)
    for u in range(N):
        for v in range(N):
            s = 0j
            for p in range(N):
                for q in range(N):
                    s += z[p, q] * np.exp(-2j * np.pi * (u * p + v * q) / N)
            ref[u, v] = s / N
    np.testing.assert_allclose(k[0] + 1j * k[1], ref, atol=1e-12)


def test_adjoint_identity_with_mask_and_coils():
    N, Nc = 16, 5
    rng = np.random.default_rng(1)
    maps = I.coil_maps(Nc, N, seed=1)
    mask = I.undersampling_mask(N, seed=1)
    x = rng.standard_normal((2, 2, N, N))
    k = rng.standard_normal((2, Nc, 2, N, N))
    lhs = np.sum(O.mri_fwd(x, maps, mask) * k)
    rhs = np.sum(x * O.mri_adj(k, maps, mask))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_pinv_inverts_a_fully_sampled_acquisition():
    N, Nc = 16, 4
    maps = I.coil_maps(Nc, N, seed=2)
    x = I.complex_phantom(3, N)[None]
    np.testing.assert_allclose(O.mri_pinv(O.mri_fwd(x, maps), maps), x, atol=1e-12)


def test_parseval_for_a_unit_modulus_coil():
    N = 16
    rng = np.random.default_rng(4)
    ph = rng.uniform(0, 2 * np.pi, (N, N))
    maps = np.stack([np.cos(ph), np.sin(ph)])[None]
    x = rng.standard_normal((1, 2, N, N))
    assert abs(np.linalg.norm(O.mri_fwd(x, maps)) - np.linalg.norm(x)) <= 1e-12 * np.linalg.norm(x)


def test_dinv_closed_form():
    N = 8
    a = np.array([0.5, 2.0, 1.5])
    maps = np.zeros((3, 2, N, N))
    maps[:, 0] = a[:, None, None] / np.sqrt(2)
    maps[:, 1] = a[:, None, None] / np.sqrt(2)
    maps[:, :, 0, 0] = 0.0
    d = O.mri_dinv(maps)
    assert d[0, 0] == 0.0
    np.testing.assert_allclose(d[1:, :], 1.0 / np.sum(a ** 2), rtol=1e-14)


def test_coil_mix_is_the_weighted_coil_sum():
    rng = np.random.default_rng(5)
    W = rng.standard_normal((3, 4)) + 1j * rng.standard_normal((3, 4))
    x = rng.standard_normal((2, 4, 2, 5, 6))
    out = O.coil_mix(W, x)
    xc = x[:, :, 0] + 1j * x[:, :, 1]
    for b in range(2):
        for j in range(3):
            ref = sum(W[j, i] * xc[b, i] for i in range(4))
            np.testing.assert_allclose(out[b, j, 0] + 1j * out[b, j, 1], ref, atol=1e-12)


def test_pca_finds_the_sources_of_rank_two_data():
    """k_c = a_c s_1 + b_c s_2: the centred covariance has rank 2, and two
    virtual coils span every coil's centred data."""
    rng = np.random.default_rng(6)
    N, Nc = 8, 6
    s = rng.standard_normal((2, N * N)) + 1j * rng.standard_normal((2, N * N))
    mix = rng.standard_normal((Nc, 2)) + 1j * rng.standard_normal((Nc, 2))
    kc = (mix @ s).reshape(Nc, N, N)
    k = np.stack([kc.real, kc.imag], axis=1)
    Q, w = O.coil_pca(k, 2)
    assert np.all(w[2:] <= 1e-10 * w[0]) and w[1] > 1e-3 * w[0]
    K = kc.reshape(Nc, -1).T
    Kb = K - K.mean(axis=0)
    np.testing.assert_allclose(Kb @ Q @ Q.conj().T, Kb, atol=1e-9 * np.abs(Kb).max())
    for l in range(2):
        i = int(np.argmax(np.abs(Q[:, l])))
        assert abs(Q[i, l].imag) <= 1e-14 and Q[i, l].real > 0


def test_coil_sketch_blocks():
    s_low = I.rademacher(np.random.default_rng(7), (3, 5))
    S = O.coil_sketch(7, 2, s_low)
    assert S.shape == (5, 7)
    np.testing.assert_array_equal(S[:2, :2], np.eye(2))
    assert np.all(S[:2, 2:] == 0) and np.all(S[2:, :2] == 0)
    assert set(np.unique(S[2:, 2:])) <= {-1.0, 1.0}


def test_csk_gradient_matches_central_differences():
    N, Nc, G = 16, 4, 2
    rng = np.random.default_rng(8)
    maps = I.coil_maps(Nc, N, seed=8)
    mask = I.undersampling_mask(N, seed=8)
    x_gt = I.complex_phantom(8, N)[None]
    y = O.mri_fwd(x_gt, maps, mask) + 0.01 * rng.standard_normal((1, Nc, 2, N, N))
    x0 = O.mri_pinv(y, maps, mask)
    g = rng.uniform(0, 360, (1, G))
    theta = 0.05 * rng.standard_normal((2, N, N))
    loss, grad, _ = O.mri_ttt_grad(theta, x0, y, maps, mask, g, 0.7)
    v = rng.standard_normal(theta.shape)
    h = 1e-3
    lp = O.mri_ttt_loss(theta + h * v, x0, y, maps, mask, g, 0.7)[0]
    lm = O.mri_ttt_loss(theta - h * v, x0, y, maps, mask, g, 0.7)[0]
    fd = (lp - lm) / (2 * h)
    assert abs(fd - np.sum(grad * v)) <= 1e-8 * abs(fd) + 1e-10
