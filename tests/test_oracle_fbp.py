"""Pins of the oracle's Ram-Lak filter H, back-projection B and B^T and
FBP = (pi/m') B H: the filter's closed-form taps and frequency response, the
exact reconstruction scale on an analytic disk, convergence on analytic
ellipse sinograms, H symmetric, B^T the transpose of B, and the exact
90-degree equivariance with numpy's rot90."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2411_05771_gb300 import inputs as I


def test_ramlak_taps():
    pi2 = math.pi ** 2
    assert O.ramlak_tap(0) == 0.25
    for n in (1, -1, 3, -3, 5, 101):
        assert abs(O.ramlak_tap(n) + 1.0 / (pi2 * n * n)) < 1e-18
    for n in (2, -2, 4, 100):
        assert O.ramlak_tap(n) == 0.0
    # a unit impulse at bin k0 returns the kernel itself, centred on k0
    nd, k0 = 31, 12
    p = np.zeros((1, nd))
    p[0, k0] = 1.0
    q = O.ramlak(p)[0]
    expect = np.array([0.25 if k == k0 else ((k - k0) % 2) * -1.0 / (pi2 * (k - k0) ** 2)
                       for k in range(nd)])
    np.testing.assert_allclose(q, expect, rtol=1e-15, atol=0)


def test_ramlak_frequency_response_is_ramp():
    """sum_n h(n) e^{-i w n} = |w|/(2 pi) on |w| <= pi for the infinite kernel
    (from sum_{odd n>0} cos(n w)/n^2 = (pi/4)(pi/2 - |w|)); the DC term is 0."""
    M = 20001
    n = np.arange(-M, M + 1)
    h = np.array([O.ramlak_tap(int(k)) for k in n])
    assert abs(h.sum()) < 1.2 / (math.pi ** 2 * M)
    for w in (0.05, 0.3, 1.0, 2.0, 3.0):
        H = np.sum(h * np.cos(w * n))
        assert abs(H - w / (2 * math.pi)) < 1e-4


def test_H_symmetric():
    rng = np.random.default_rng(0)
    p, q = rng.standard_normal((2, 5, 41))
    assert abs(np.sum(O.ramlak(p) * q) - np.sum(p * O.ramlak(q))) < 1e-12


@pytest.mark.parametrize("N", [16, 17])
def test_backproject_adjoint_identity(N):
    nd = O.ndet(N)
    rng = np.random.default_rng(N)
    angs = np.concatenate([[0.0, 45.0, 90.0], rng.uniform(0, 360, 15)])
    q = rng.standard_normal((angs.size, nd))
    x = rng.standard_normal((N, N))
    lhs = np.sum(O.backproject(q, angs, N) * x)
    rhs = np.sum(q * O.backproject_adj(x, angs, nd))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1)


def test_backproject_explicit_transpose():
    N, nd = 8, 13
    angs = np.arange(12) * 15.0
    Bm = np.stack([O.backproject(e.reshape(12, nd), angs, N).ravel()
                   for e in np.eye(12 * nd)], axis=1)
    Bt = np.stack([O.backproject_adj(e.reshape(N, N), angs, nd).ravel()
                   for e in np.eye(N * N)], axis=1)
    np.testing.assert_allclose(Bt, Bm.T, rtol=0, atol=1e-15)


def test_backproject_constant_row():
    """Back-projecting a constant sinogram adds the constant once per angle."""
    N = 20
    nd = O.ndet(N)
    angs = np.arange(0.0, 180.0, 10.0)
    x = O.backproject(np.full((angs.size, nd), 2.5), angs, N)
    np.testing.assert_allclose(x, 2.5 * angs.size, rtol=1e-14)


@pytest.mark.parametrize("N", [64, 128])
def test_fbp_reconstructs_disk(N):
    """FBP of the exact line integrals of a unit disk gives ~1 inside, ~0
    outside: pins the filter's scale and the pi/m' factor."""
    nd = O.ndet(N)
    n_ang = 2 * N
    angs = I.uniform_angles(n_ang)
    R = 0.5 * N / 2
    rec = O.fbp(I.disk_sinogram(R, n_ang, nd), angs, N)
    c = np.arange(N) - (N - 1) / 2
    r = np.hypot(c[None, :], c[:, None])
    inner = rec[r < 0.8 * R]
    outer = rec[(r > 1.25 * R) & (r < 0.45 * N)]
    assert abs(inner.mean() - 1.0) < 0.01
    assert np.abs(inner - 1.0).max() < 0.05
    assert abs(outer.mean()) < 0.01


def test_fbp_ellipses_converge():
    e = I.random_ellipses(3)
    ps = []
    for N in (64, 128):
        nd = O.ndet(N)
        angs = I.uniform_angles(2 * N)
        rec = O.fbp(I.analytic_sinogram(e, N, angs, nd), angs, N)
        ps.append(O.psnr(rec, I.rasterize(e, N, supersample=2)))
    assert ps[1] > ps[0] > 18.0


def test_fbp_rot90_equivariance():
    """FBP(p shifted by 90 degrees) = T_90 FBP(p) with T_90 = numpy's rot90."""
    N = 24
    nd = O.ndet(N)
    n_ang = 36
    angs = I.uniform_angles(n_ang)
    p = np.random.default_rng(1).standard_normal((n_ang, nd))
    half = n_ang // 2
    shifted = np.concatenate([p[half:, ::-1], p[:half]], axis=0)
    np.testing.assert_allclose(O.fbp(shifted, angs, N), np.rot90(O.fbp(p, angs, N)),
                               atol=1e-12)


def test_sketched_fbp_uses_sketch_size():
    """A_S^dagger over m angles scales by pi/m: FBP of a constant-in-angle
    sinogram is independent of how many (equally spaced) angles are used."""
    N = 32
    nd = O.ndet(N)
    R = 0.4 * N / 2
    full = I.uniform_angles(64)
    rec_full = O.fbp(I.disk_sinogram(R, 64, nd), full, N)
    idx = I.sketch_indices(64, 16, 3)
    rec_sk = O.fbp(I.disk_sinogram(R, 16, nd), O.select(full, idx), N)
    c = np.arange(N) - (N - 1) / 2
    r = np.hypot(c[None, :], c[:, None])
    assert abs(rec_sk[r < 0.6 * R].mean() - rec_full[r < 0.6 * R].mean()) < 0.02
