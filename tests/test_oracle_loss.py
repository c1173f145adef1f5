"""Pins of the oracle's EI / SkEI loss composition (Eq. e:skeiloss,
Eq. e:skeilossttt, Algorithm 2), its hand-written gradient and Adam.

With the stand-in network F(u) = u + theta every operator is linear, so the
loss is an exact quadratic in theta and a central finite difference equals
the derivative up to rounding for any step h: the gradient is pinned by
forward evaluations alone.  Adam is pinned against torch.optim.Adam."""
import numpy as np
import pytest

import oracle as O
from paper_2411_05771_gb300 import inputs as I


def _problem(seed=0, N=12, n_ang=12, m=4, B=2, G=3):
    rng = np.random.default_rng(seed)
    nd = O.ndet(N)
    angs = I.uniform_angles(n_ang)
    x0 = rng.random((B, N, N))
    theta = 0.1 * rng.standard_normal((N, N))
    y = rng.random((B, n_ang, nd)) * 5
    g = I.rotation_angles(rng, B, G)
    idx = I.sketch_indices(n_ang, m, int(rng.integers(0, n_ang // m)))
    return dict(N=N, nd=nd, angs=angs, x0=x0, theta=theta, y=y, g=g, idx=idx)


def test_mc_vanishes_on_consistent_data():
    """y = A x1 exactly gives a zero (sketched) residual: the sketch selects
    the same rows of y as of A."""
    P = _problem()
    x1 = P["x0"]
    y = O.proj_fwd(x1, P["angs"], P["nd"])
    for mc_idx in (None, P["idx"]):
        r, _, _ = O.ei_stage1(x1, y, P["angs"], mc_idx, P["idx"], P["g"])
        assert np.count_nonzero(r) == 0


def test_full_sketch_equals_plain_ei():
    P = _problem(1)
    x1 = P["x0"] + P["theta"]
    a = O.ei_stage1(x1, P["y"], P["angs"], None, None, P["g"])
    b = O.ei_stage1(x1, P["y"], P["angs"], np.arange(12), np.arange(12), P["g"])
    for u, v in zip(a, b):
        np.testing.assert_array_equal(u, v)


def test_loss_parts():
    P = _problem(2)
    args = (P["theta"], P["x0"], P["y"], P["angs"], P["idx"], P["idx"], P["g"])
    l0, t0 = O.ttt_loss(*args, 0.0, 2.0)
    np.testing.assert_allclose(l0, np.mean(t0["mc"]), rtol=1e-15)
    np.testing.assert_allclose(t0["mc"], 2.0 * np.sum(t0["r"] ** 2, axis=(1, 2)), rtol=1e-14)
    l1, t1 = O.ttt_loss(*args, 0.5, 2.0)
    B, G = P["g"].shape
    np.testing.assert_allclose(l1 - l0, 0.5 / (B * G) * t1["ei"].sum(), rtol=1e-12)
    # x3 = z + theta, x2 = T_g x1: the EI term is the rotated output against
    # the re-measured and re-reconstructed one
    np.testing.assert_allclose(t1["x3"], t1["z"] + P["theta"], rtol=0, atol=0)


@pytest.mark.parametrize("sketched", [False, True])
def test_gradient_matches_central_differences(sketched):
    P = _problem(3)
    idx = P["idx"] if sketched else None
    lam, mcs = 0.7, (3.0 if sketched else 1.0)
    args = (P["x0"], P["y"], P["angs"], idx, idx, P["g"], lam, mcs)
    loss, grad, _ = O.ttt_grad(P["theta"], *args)
    rng = np.random.default_rng(9)
    h = 1e-3
    N = P["N"]
    pix = rng.choice(N * N, 24, replace=False)
    for q in pix:
        e = np.zeros(N * N)
        e[q] = h
        e = e.reshape(N, N)
        lp, _ = O.ttt_loss(P["theta"] + e, *args)
        lm, _ = O.ttt_loss(P["theta"] - e, *args)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - grad.ravel()[q]) <= 1e-7 * np.abs(grad).max()
    # one random direction covers every pixel at once
    v = rng.standard_normal((N, N))
    lp, _ = O.ttt_loss(P["theta"] + h * v, *args)
    lm, _ = O.ttt_loss(P["theta"] - h * v, *args)
    assert abs((lp - lm) / (2 * h) - np.sum(grad * v)) <= 1e-8 * abs(np.sum(grad * v)) + 1e-9


def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(4)
    theta = rng.standard_normal((5, 7))
    p = torch.nn.Parameter(torch.tensor(theta, dtype=torch.float64))
    opt = torch.optim.Adam([p], lr=5e-4, betas=(0.9, 0.999), eps=1e-8)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    for step in range(1, 8):
        g = rng.standard_normal(theta.shape)
        p.grad = torch.tensor(g)
        opt.step()
        theta, m, v = O.adam_step(theta, g, m, v, step)
        np.testing.assert_allclose(theta, p.detach().numpy(), rtol=1e-13, atol=1e-15)


def test_psnr_definition():
    ref = np.array([[0.0, 1.0], [2.0, 3.0]])
    x = ref + 0.1
    assert abs(O.psnr(x, ref) - 10 * np.log10(9.0 / 0.01)) < 1e-12


def _rows(n_ang, m, B, seed):
    rng = np.random.default_rng(seed)
    return np.stack([I.sketch_indices(n_ang, m, int(rng.integers(0, n_ang // m)))
                     for _ in range(B)])


def test_per_sample_sketches_with_equal_rows_are_the_shared_sketch():
    """Algorithm 1 with the same sketch drawn for every measurement is the
    shared-sketch loss and gradient."""
    P = _problem(5, B=3)
    rows = np.stack([P["idx"]] * 3)
    args = (P["x0"], P["y"], P["angs"])
    for mc in (None, "sk"):
        l1, g1, _ = O.ttt_grad(P["theta"], *args, P["idx"] if mc else None, P["idx"], P["g"],
                               0.7, 2.0)
        l2, g2, _ = O.ttt_grad_per_sample(P["theta"], *args, rows if mc else None, rows, P["g"],
                                          0.7, 2.0)
        assert abs(l1 - l2) <= 1e-12 * abs(l1)
        np.testing.assert_allclose(g2, g1, rtol=0, atol=1e-12 * np.abs(g1).max())


@pytest.mark.parametrize("mc_rows", [False, True])
def test_per_sample_gradient_matches_central_differences(mc_rows):
    """Distinct sketches per measurement: the hand-written gradient (with
    each measurement's MC coefficient mc_scale / B) against finite
    differences of the loss (exact: the loss is quadratic in theta)."""
    P = _problem(6, B=3, G=2)
    rows = _rows(len(P["angs"]), 4, 3, seed=7)
    assert len({tuple(r) for r in rows}) > 1
    args = (P["x0"], P["y"], P["angs"], rows if mc_rows else None, rows, P["g"], 0.7, 3.0)
    loss, grad, _ = O.ttt_grad_per_sample(P["theta"], *args)
    rng = np.random.default_rng(8)
    h = 1e-3
    v = rng.standard_normal(P["theta"].shape)
    lp, _ = O.ttt_loss_per_sample(P["theta"] + h * v, *args)
    lm, _ = O.ttt_loss_per_sample(P["theta"] - h * v, *args)
    assert abs((lp - lm) / (2 * h) - np.sum(grad * v)) <= 1e-8 * abs(np.sum(grad * v)) + 1e-9
    # and the loss is the mean of the single-measurement losses
    parts = [O.ttt_loss(P["theta"], P["x0"][b:b + 1], P["y"][b:b + 1], P["angs"],
                        rows[b] if mc_rows else None, rows[b], P["g"][b:b + 1], 0.7, 3.0)[0]
             for b in range(3)]
    assert abs(loss - np.mean(parts)) <= 1e-12 * abs(loss)
