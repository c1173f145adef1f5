"""Pins of the oracle's geometry, Joseph projector A and its adjoint A^T
against what mathematics fixes independently of the oracle's own loops:
closed forms at 0 and 90 degrees, chord lengths, the continuous Radon
transform of disks and ellipses, exact 90/180-degree symmetries (with numpy's
rot90 as the rotation), the transpose relation on an explicit 8x8 matrix."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2411_05771_gb300 import inputs as I


def test_ndet_rule():
    # the detector sizes quoted for the 64/256/512 workloads
    assert (O.ndet(64), O.ndet(256), O.ndet(512)) == (91, 363, 725)
    assert O.ndet(8) == 13
    for N in range(1, 700):
        k = O.ndet(N)
        assert k % 2 == 1 and k >= N * math.sqrt(2) and k - 2 < N * math.sqrt(2)


def test_trig_reduction():
    for q in range(-4, 9):
        c, s = O.trig(90.0 * q)
        assert (c, s) == ({0: 1.0, 1: 0.0, 2: -1.0, 3: 0.0}[q % 4],
                          {0: 0.0, 1: 1.0, 2: 0.0, 3: -1.0}[q % 4])
    rng = np.random.default_rng(0)
    for deg in rng.uniform(-400, 400, 200):
        c, s = O.trig(deg)
        assert abs(c - math.cos(math.radians(deg))) < 1e-14
        assert abs(s - math.sin(math.radians(deg))) < 1e-14


def test_mode_rule():
    assert O.row_mode(0.0) and O.row_mode(45.0) and O.row_mode(135.0 + 1e-9)
    assert not O.row_mode(45.0 + 1e-9) and not O.row_mode(90.0) and not O.row_mode(135.0)
    assert O.row_mode(180.0) and O.row_mode(225.0) and not O.row_mode(270.0)


def _hat(d):
    return np.clip(1.0 - np.abs(d), 0.0, None)


@pytest.mark.parametrize("N", [8, 9, 32, 33])
def test_theta0_is_interpolated_column_sums(N):
    """At 0 degrees the ray x = u_k meets every row at column c = u_k +
    (N-1)/2, so p_k = sum_j hat(j - c) colsum_j (half-pixel shifts for even N)."""
    nd = O.ndet(N)
    x = np.random.default_rng(N).random((N, N))
    p = O.proj_fwd(x, [0.0], nd)[0]
    u = np.arange(nd) - (nd - 1) / 2
    cpos = u + (N - 1) / 2
    expect = np.array([np.sum(_hat(np.arange(N) - c) * x.sum(axis=0)) for c in cpos])
    np.testing.assert_allclose(p, expect, rtol=0, atol=1e-12)


@pytest.mark.parametrize("N", [8, 9, 32])
def test_theta90_is_interpolated_row_sums_y_up(N):
    """At 90 degrees the ray y = u_k meets row (N-1)/2 - u_k: large bins see
    the TOP rows (y points up)."""
    nd = O.ndet(N)
    x = np.random.default_rng(N + 1).random((N, N))
    p = O.proj_fwd(x, [90.0], nd)[0]
    u = np.arange(nd) - (nd - 1) / 2
    rpos = (N - 1) / 2 - u
    expect = np.array([np.sum(_hat(np.arange(N) - r) * x.sum(axis=1)) for r in rpos])
    np.testing.assert_allclose(p, expect, rtol=0, atol=1e-12)
    # a single bright top row only lights bins with u > 0
    top = np.zeros((N, N))
    top[0] = 1.0
    q = O.proj_fwd(top, [90.0], nd)[0]
    assert q[u > 0].sum() > 0 and q[u < -0.5].sum() == 0


@pytest.mark.parametrize("deg", [0.0, 20.0, 45.0, 60.0, 90.0, 120.0, 135.0, 170.0])
def test_constant_image_gives_chord_length(deg):
    """A applied to the all-ones image equals the length of the ray inside
    the square spanned by the pixel centres, for rays that cross every line
    of the walking direction within it (N/|cos| in row mode, N/|sin| in
    column mode)."""
    N = 32
    nd = O.ndet(N)
    p = O.proj_fwd(np.ones((N, N)), [deg], nd)[0]
    c, s = math.cos(math.radians(deg)), math.sin(math.radians(deg))
    u = np.arange(nd) - (nd - 1) / 2
    h = (N - 1) / 2
    row = O.row_mode(deg)
    w = 1 / abs(c) if row else 1 / abs(s)
    # in row mode the crossing column of row y is (u - y s)/c; interior if it
    # stays within [-h, h] for y = +-h
    if row:
        inside = np.maximum(np.abs((u - h * s) / c), np.abs((u + h * s) / c)) <= h
    else:
        inside = np.maximum(np.abs((u - h * c) / s), np.abs((u + h * c) / s)) <= h
    assert inside.sum() >= 1
    np.testing.assert_allclose(p[inside], N * w, rtol=1e-13)


def test_disk_radon_convergence():
    """Centred uniform disk of physical radius 0.6: line integral 2 sqrt(R^2-u^2)."""
    angs = [0.0, 17.0, 30.0, 45.0, 60.0, 90.0, 112.0, 135.0, 150.0]
    errs = []
    for N in (32, 64, 128):
        nd = O.ndet(N)
        R = 0.6 * N / 2
        e = I.Ellipses(*(np.array([v]) for v in (0.0, 0.0, 0.6, 0.6, 0.0, 1.0)))
        x = I.rasterize(e, N, supersample=4)
        p = O.proj_fwd(x, angs, nd)
        ref = I.disk_sinogram(R, len(angs), nd)
        errs.append(np.linalg.norm(p - ref) / np.linalg.norm(ref))
    assert errs[2] < errs[1] < errs[0]
    assert errs[2] < 6e-3


def test_ellipse_radon_convergence():
    """Random off-centre, rotated ellipses: the discrete sinogram converges to
    the analytic Radon transform (pins angle sign, detector direction and
    centring)."""
    e = I.random_ellipses(7)
    angs = np.arange(0.0, 180.0, 7.5)
    errs = []
    for N in (32, 64, 128):
        nd = O.ndet(N)
        x = I.rasterize(e, N, supersample=4)
        p = O.proj_fwd(x, angs, nd)
        ref = I.analytic_sinogram(e, N, angs, nd)
        errs.append(np.linalg.norm(p - ref) / np.linalg.norm(ref))
    assert errs[2] < errs[1] < errs[0]
    assert errs[2] < 2e-2


def test_offcentre_point_trace():
    """A small disk at physical (0.5, 0.2) projects to u = (N/2)(0.5 cos t +
    0.2 sin t) at every angle t."""
    N = 64
    nd = O.ndet(N)
    e = I.Ellipses(*(np.array([v]) for v in (0.5, 0.2, 0.06, 0.06, 0.0, 1.0)))
    x = I.rasterize(e, N, supersample=4)
    angs = np.arange(0.0, 360.0, 15.0)
    p = O.proj_fwd(x, angs, nd)
    u = np.arange(nd) - (nd - 1) / 2
    centroid = (p * u).sum(axis=1) / p.sum(axis=1)
    t = np.radians(angs)
    expect = (N / 2) * (0.5 * np.cos(t) + 0.2 * np.sin(t))
    np.testing.assert_allclose(centroid, expect, atol=0.05)


def _explicit(fn, n_in, shape_in):
    cols = []
    for q in range(n_in):
        e = np.zeros(n_in)
        e[q] = 1.0
        cols.append(fn(e.reshape(shape_in)).ravel())
    return np.stack(cols, axis=1)


def test_explicit_8x8_matrix_transpose():
    """N=8, 13 bins, 12 angles including 0/45/90/135: the adjoint's scatter
    loop gives exactly the transpose of the forward loop's matrix."""
    N, nd = 8, 13
    angs = np.arange(12) * 15.0
    A = _explicit(lambda v: O.proj_fwd(v, angs, nd), N * N, (N, N))
    At = _explicit(lambda v: O.proj_adj(v, angs, N), 12 * nd, (12, nd))
    np.testing.assert_allclose(At, A.T, rtol=0, atol=1e-14)
    assert np.array_equal(At != 0, A.T != 0)
    assert A.min() >= 0.0
    # every sample spreads a weight of exactly 1 over at most 2 pixels of one
    # line: rows of A sum to W * (number of in-image samples)
    assert np.count_nonzero(A) > 0


@pytest.mark.parametrize("N", [16, 17])
def test_adjoint_identity(N):
    nd = O.ndet(N)
    rng = np.random.default_rng(N)
    angs = np.concatenate([[0.0, 45.0, 90.0, 135.0], rng.uniform(0, 360, 20)])
    x = rng.standard_normal((N, N))
    y = rng.standard_normal((angs.size, nd))
    lhs = np.sum(O.proj_fwd(x, angs, nd) * y)
    rhs = np.sum(x * O.proj_adj(y, angs, N))
    assert abs(lhs - rhs) <= 1e-12 * (abs(lhs) + 1)


@pytest.mark.parametrize("N", [16, 17])
def test_rot90_sinogram_shift(N):
    """A(T_90 x)[t] = A(x)[t - 90]; rows that wrap below 0 come from t + 90
    with the detector flipped.  T_90 here is numpy's rot90 (counter-clockwise),
    independent of the oracle's rotation."""
    nd = O.ndet(N)
    n_ang = 24  # 7.5 degree steps: 90 degrees is 12 rows
    angs = 180.0 * np.arange(n_ang) / n_ang
    x = np.random.default_rng(3).random((N, N))
    p = O.proj_fwd(x, angs, nd)
    pr = O.proj_fwd(np.rot90(x), angs, nd)
    half = n_ang // 2
    np.testing.assert_allclose(pr[half:], p[:half], atol=1e-12)
    np.testing.assert_allclose(pr[:half], p[half:, ::-1], atol=1e-12)


def test_180_flip():
    N = 20
    nd = O.ndet(N)
    rng = np.random.default_rng(4)
    base = rng.uniform(0, 180, 10)
    x = rng.random((N, N))
    p0 = O.proj_fwd(x, base, nd)
    p1 = O.proj_fwd(x, base + 180.0, nd)
    np.testing.assert_allclose(p1, p0[:, ::-1], atol=1e-11)


def test_sketch_rows_are_rows_of_A():
    N = 16
    nd = O.ndet(N)
    angs = I.uniform_angles(12)
    idx = I.sketch_indices(12, 4, 2)
    x = np.random.default_rng(5).random((N, N))
    full = O.proj_fwd(x, angs, nd)
    sk = O.proj_fwd(x, O.select(angs, idx), nd)
    np.testing.assert_array_equal(sk, full[idx])
    assert list(idx) == [2, 5, 8, 11]
