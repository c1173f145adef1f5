"""Pins of the oracle's bilinear rotation T_g and its scatter adjoint:
identity at 0, exact permutations equal to numpy's rot90 at multiples of 90,
direction and centre on an analytic Gaussian, the transpose relation, and the
continuous identity R(T_g f)(t) = R f(t - g) linking rotation and projection."""
import math

import numpy as np
import pytest

import oracle as O


def test_rotate_zero_is_identity():
    x = np.random.default_rng(0).random((17, 17))
    np.testing.assert_array_equal(O.rotate(x, 0.0), x)
    np.testing.assert_array_equal(O.rotate(x, 360.0), x)


@pytest.mark.parametrize("N", [8, 9, 16])
def test_rotate_quarter_turns_are_rot90(N):
    x = np.random.default_rng(N).random((N, N))
    for k in (1, 2, 3, -1):
        np.testing.assert_array_equal(O.rotate(x, 90.0 * k), np.rot90(x, k))


def _gauss(N, x0, y0, sig):
    X = (np.arange(N) - (N - 1) / 2)[None, :]
    Y = ((N - 1) / 2 - np.arange(N))[:, None]
    return np.exp(-((X - x0) ** 2 + (Y - y0) ** 2) / (2 * sig * sig))


@pytest.mark.parametrize("g", [30.0, 137.0, 251.5])
def test_rotate_moves_blob_counter_clockwise(g):
    """An off-centre Gaussian at (10, 4) moves to R(g)(10, 4)."""
    N = 64
    x = _gauss(N, 10.0, 4.0, 4.0)
    t = math.radians(g)
    x1, y1 = 10 * math.cos(t) - 4 * math.sin(t), 10 * math.sin(t) + 4 * math.cos(t)
    # bilinear error is at most ~h^2 |f''| / 4 ~ 0.016 here; a rotation the
    # wrong way or about the wrong centre is off by O(1)
    np.testing.assert_allclose(O.rotate(x, g), _gauss(N, x1, y1, 4.0), atol=0.025)


@pytest.mark.parametrize("N", [12, 13])
def test_rotate_adjoint_identity(N):
    rng = np.random.default_rng(N)
    for g in rng.uniform(0, 360, 6):
        a, b = rng.standard_normal((2, N, N))
        lhs = np.sum(O.rotate(a, g) * b)
        rhs = np.sum(a * O.rotate_adj(b, g))
        assert abs(lhs - rhs) < 1e-12 * (abs(lhs) + 1)


def test_rotate_explicit_transpose():
    N = 6
    g = 33.0
    T = np.stack([O.rotate(e.reshape(N, N), g).ravel() for e in np.eye(N * N)], axis=1)
    Tt = np.stack([O.rotate_adj(e.reshape(N, N), g).ravel() for e in np.eye(N * N)], axis=1)
    np.testing.assert_allclose(Tt, T.T, rtol=0, atol=1e-15)


def test_rotation_shifts_sinogram():
    """Projection of the rotated image at angle t equals the projection of the
    image at t - g (up to interpolation error for a smooth object)."""
    N = 64
    nd = O.ndet(N)
    x = _gauss(N, 8.0, -5.0, 4.0) + 0.5 * _gauss(N, -6.0, 3.0, 6.0)
    g = 40.0
    angs = np.arange(0.0, 180.0, 10.0)
    lhs = O.proj_fwd(O.rotate(x, g), angs, nd)
    rhs = O.proj_fwd(x, angs - g, nd)
    assert np.linalg.norm(lhs - rhs) / np.linalg.norm(rhs) < 5e-3
