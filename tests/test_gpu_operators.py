"""GPU parity of the operator kernels (A, A^T, H, B, B^T, FBP, T_g, T_g^T)
against the FP64 oracle, through the C ABI.

Tolerances (FP32 storage, FP32 arithmetic): rel-L2 <= 1e-5 elementwise over
the whole output; adjoint mismatch |<Ax,y> - <x,A^T y>| / (||Ax|| ||y||)
<= 1e-6 with FP64 inner products; BF16 storage: rel-L2 <= 1e-2 against the
oracle run on the same BF16-rounded inputs."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2411_05771_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5
ADJ_TOL = 1e-6
BF16_TOL = 1e-2


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


def phantoms(B, N, seed0=0):
    return np.stack([I.rasterize(I.random_ellipses(seed0 + b), N) for b in range(B)])


# (N, n_angles, B, m): config 1 (64^2, 60 x 91, B=1), config 2 (8 x 256^2,
# 180 x 363, sketch 45), ragged sizes that leave partial tiles/bands, tiny N
CASES = [(64, 60, 1, 60), (64, 60, 1, 15), (256, 180, 8, 180), (256, 180, 8, 45),
         (37, 24, 3, 8), (100, 30, 2, 10), (8, 12, 2, 12), (5, 7, 1, 7)]


def _idx(n_ang, m, seed):
    if m == n_ang:
        return None
    off = I.random_sketch_offset(np.random.default_rng(seed), n_ang, m)
    return I.sketch_indices(n_ang, m, off)


@pytest.mark.parametrize("N,n_ang,B,m", CASES)
def test_proj_fwd_and_residual(S, N, n_ang, B, m):
    plan = S.Plan(N, n_ang)
    x = phantoms(B, N) + 0.1 * np.random.default_rng(N).standard_normal((B, N, N))
    idx = _idx(n_ang, m, N)
    angs = O.select(plan.angles_deg, idx)
    ref = O.proj_fwd(x, angs, plan.n_det)
    idx_d = None if idx is None else dev(idx, torch.int32)
    got = S.proj_fwd(plan, dev(x), idx_d)
    assert rel(host(got), ref) <= FP32_TOL
    y = O.proj_fwd(phantoms(B, N, 100), plan.angles_deg, plan.n_det)
    got_r = S.proj_fwd(plan, dev(x), idx_d, y=dev(y))
    y_s = y if idx is None else y[:, idx]
    # a residual is a difference of larger quantities: its FP32 error is
    # bounded relative to the operands, not to itself
    assert np.linalg.norm(host(got_r) - (y_s - ref)) <= FP32_TOL * np.linalg.norm(y_s)
    assert plan.status() == 0


@pytest.mark.parametrize("N,n_ang,B,m", CASES)
def test_proj_adj(S, N, n_ang, B, m):
    plan = S.Plan(N, n_ang)
    rng = np.random.default_rng(N + 1)
    idx = _idx(n_ang, m, N + 1)
    angs = O.select(plan.angles_deg, idx)
    p = rng.standard_normal((B, m, plan.n_det))
    ref = O.proj_adj(p, angs, N)
    idx_d = None if idx is None else dev(idx, torch.int32)
    got = S.proj_adj(plan, dev(p), idx_d)
    assert rel(host(got), ref) <= FP32_TOL
    # accumulate form alpha A^T p + beta x
    x0 = rng.standard_normal((B, N, N))
    out = dev(x0)
    S.proj_adj(plan, dev(p), idx_d, alpha=-0.5, beta=2.0, out=out)
    assert rel(host(out), -0.5 * ref + 2.0 * x0) <= FP32_TOL


@pytest.mark.parametrize("N,n_ang", [(64, 60), (33, 20), (256, 180)])
def test_adjoint_identity(S, N, n_ang):
    plan = S.Plan(N, n_ang)
    rng = np.random.default_rng(5)
    x = dev(rng.standard_normal((2, N, N)))
    y = dev(rng.standard_normal((2, n_ang, plan.n_det)))
    Ax = S.proj_fwd(plan, x)
    Aty = S.proj_adj(plan, y)
    lhs = float((Ax.double() * y.double()).sum())
    rhs = float((x.double() * Aty.double()).sum())
    scale = float(Ax.double().norm() * y.double().norm())
    assert abs(lhs - rhs) / scale <= ADJ_TOL
    # the same for B and B^T
    q = S.backproject(plan, y)
    Btx = S.backproject_adj(plan, x)
    lhs = float((q.double() * x.double()).sum())
    rhs = float((y.double() * Btx.double()).sum())
    assert abs(lhs - rhs) / float(q.double().norm() * x.double().norm()) <= ADJ_TOL


def _unit_columns(fn, n_in, shape_in):
    eye = torch.eye(n_in, device="cuda", dtype=torch.float32).reshape((n_in,) + shape_in)
    return torch.stack([fn(eye[q:q + 1]).reshape(-1) for q in range(n_in)], dim=1)


def test_explicit_8x8_transposes_are_bitwise(S):
    """N=8, 13 bins, 12 angles including 0/45/90/135: the gathered adjoints
    reproduce the forward weights bit for bit, and both match the oracle."""
    N, n_ang = 8, 12
    angs = np.arange(n_ang) * 15.0
    plan = S.Plan(N, n_ang, angs)
    nd = plan.n_det
    A = _unit_columns(lambda v: S.proj_fwd(plan, v), N * N, (N, N))
    At = _unit_columns(lambda v: S.proj_adj(plan, v), n_ang * nd, (n_ang, nd))
    assert torch.equal(At, A.t())
    A_ref = np.stack([O.proj_fwd(e.reshape(N, N), angs, nd).ravel() for e in np.eye(N * N)], 1)
    assert np.abs(host(A) - A_ref).max() <= 1e-5
    Bm = _unit_columns(lambda v: S.backproject(plan, v), n_ang * nd, (n_ang, nd))
    Bt = _unit_columns(lambda v: S.backproject_adj(plan, v), N * N, (N, N))
    assert torch.equal(Bt, Bm.t())
    B_ref = np.stack([O.backproject(e.reshape(n_ang, nd), angs, N).ravel()
                      for e in np.eye(n_ang * nd)], 1)
    assert np.abs(host(Bm) - B_ref).max() <= 1e-5
    for g in (33.0, 90.0, 217.5):
        gd = torch.tensor([[g]], dtype=torch.float64, device="cuda")
        T = _unit_columns(lambda v: S.rotate(v, gd)[:, 0], N * N, (N, N))
        Tt = _unit_columns(lambda v: S.rotate_adj(v[:, None], gd), N * N, (N, N))
        assert torch.equal(Tt, T.t())


@pytest.mark.parametrize("N,n_ang,B,m", CASES)
def test_filter_backproject_fbp(S, N, n_ang, B, m):
    plan = S.Plan(N, n_ang)
    rng = np.random.default_rng(N + 2)
    idx = _idx(n_ang, m, N + 2)
    angs = O.select(plan.angles_deg, idx)
    idx_d = None if idx is None else dev(idx, torch.int32)
    p = rng.standard_normal((B, m, plan.n_det))
    assert rel(host(S.filter(plan, dev(p), 0.75)), 0.75 * O.ramlak(p)) <= FP32_TOL
    assert rel(host(S.backproject(plan, dev(p), idx_d)), O.backproject(p, angs, N)) <= FP32_TOL
    x = rng.standard_normal((B, N, N))
    assert rel(host(S.backproject_adj(plan, dev(x), idx_d)),
               O.backproject_adj(x, angs, plan.n_det)) <= FP32_TOL
    assert rel(host(S.fbp(plan, dev(p), idx_d)), O.fbp(p, angs, N)) <= FP32_TOL
    assert rel(host(S.fbp_adj(plan, dev(x), idx_d)), O.fbp_adj(x, angs, plan.n_det)) <= FP32_TOL


@pytest.mark.parametrize("N,B,G", [(64, 1, 4), (256, 2, 4), (37, 3, 2), (8, 1, 5),
                                   (512, 1, 4)])   # the 512^2 step's rotations
def test_rotate_and_transpose(S, N, B, G):
    rng = np.random.default_rng(N)
    x = rng.standard_normal((B, N, N))
    g = I.rotation_angles(rng, B, G)
    gd = dev(g, torch.float64)
    got = S.rotate(dev(x), gd)
    assert rel(host(got), O.rotate_batch(x, g)) <= FP32_TOL
    gout = rng.standard_normal((B, G, N, N))
    got_t = S.rotate_adj(dev(gout), gd)
    assert rel(host(got_t), O.rotate_adj_batch(gout, g)) <= FP32_TOL


def test_quarter_turns_are_exact(S):
    x = torch.randn(2, 37, 37, device="cuda")
    for k in (1, 2, 3, -1):
        gd = torch.full((2, 1), 90.0 * k, dtype=torch.float64, device="cuda")
        assert torch.equal(S.rotate(x, gd)[:, 0], torch.rot90(x, k, dims=(1, 2)))


def test_rot90_sinogram_shift_on_gpu(S):
    """A(T_90 x)[t] = A(x)[t - 90] with wrap-around flip (24 angles)."""
    N, n_ang = 48, 24
    plan = S.Plan(N, n_ang)
    x = torch.randn(1, N, N, device="cuda")
    p = host(S.proj_fwd(plan, x))[0]
    pr = host(S.proj_fwd(plan, torch.rot90(x, 1, dims=(1, 2)).contiguous()))[0]
    h = n_ang // 2
    assert rel(pr[h:], p[:h]) <= FP32_TOL
    assert rel(pr[:h], p[h:, ::-1]) <= FP32_TOL


def test_angles_at_mode_boundaries_and_unusual_values(S):
    N = 40
    angs = np.array([45.0, 135.0, 44.9999, 135.0001, -30.0, 400.0, 225.0, 0.0, 90.0, 180.0])
    plan = S.Plan(N, angs.size, angs)
    x = np.random.default_rng(2).random((1, N, N))
    assert rel(host(S.proj_fwd(plan, dev(x))), O.proj_fwd(x, angs, plan.n_det)) <= FP32_TOL
    p = np.random.default_rng(3).standard_normal((1, angs.size, plan.n_det))
    assert rel(host(S.proj_adj(plan, dev(p))), O.proj_adj(p, angs, N)) <= FP32_TOL


def test_custom_detector_sizes(S):
    # a short even detector (rays clipped) and a long one
    for nd in (40, 120):
        N, n_ang = 50, 16
        plan = S.Plan(N, n_ang, n_det=nd)
        assert plan.n_det == nd
        x = np.random.default_rng(nd).random((2, N, N))
        assert rel(host(S.proj_fwd(plan, dev(x))), O.proj_fwd(x, plan.angles_deg, nd)) <= FP32_TOL
        p = np.random.default_rng(nd + 1).standard_normal((2, n_ang, nd))
        assert rel(host(S.proj_adj(plan, dev(p))), O.proj_adj(p, plan.angles_deg, N)) <= FP32_TOL
        assert rel(host(S.fbp(plan, dev(p))), O.fbp(p, plan.angles_deg, N)) <= FP32_TOL


def test_bad_angle_index_is_reported_not_read(S):
    N, n_ang = 32, 10
    plan = S.Plan(N, n_ang)
    x = dev(np.random.default_rng(0).random((1, N, N)))
    idx = torch.tensor([1, 99, 3], dtype=torch.int32, device="cuda")
    out = S.proj_fwd(plan, x, idx)
    assert plan.status(reset=True) & 1
    o = host(out)[0]
    assert np.all(o[1] == 0) and np.abs(o[0]).sum() > 0
    assert plan.status() == 0


@pytest.mark.parametrize("N,n_ang,B,m", [(64, 60, 1, 60), (256, 180, 2, 45)])
def test_bf16_storage(S, N, n_ang, B, m):
    plan = S.Plan(N, n_ang)
    idx = _idx(n_ang, m, 7)
    angs = O.select(plan.angles_deg, idx)
    idx_d = None if idx is None else dev(idx, torch.int32)
    xb = dev(phantoms(B, N), torch.bfloat16)
    x64 = host(xb)
    assert rel(host(S.proj_fwd(plan, xb, idx_d)), O.proj_fwd(x64, angs, plan.n_det)) <= BF16_TOL
    pb = dev(np.random.default_rng(1).standard_normal((B, m, plan.n_det)), torch.bfloat16)
    p64 = host(pb)
    assert rel(host(S.proj_adj(plan, pb, idx_d)), O.proj_adj(p64, angs, N)) <= BF16_TOL
    assert rel(host(S.fbp(plan, pb, idx_d)), O.fbp(p64, angs, N)) <= BF16_TOL
    g = I.rotation_angles(np.random.default_rng(2), B, 3)
    assert rel(host(S.rotate(xb, dev(g, torch.float64))), O.rotate_batch(x64, g)) <= BF16_TOL


def test_batched_jobs_match_single_calls(S):
    """Two image sets with different angle subsets and storage types in one
    launch give what separate calls give."""
    N, n_ang = 96, 40
    plan = S.Plan(N, n_ang)
    rng = np.random.default_rng(8)
    x1 = dev(rng.random((2, N, N)))
    x2 = dev(rng.random((3, N, N)), torch.bfloat16)
    y = dev(rng.random((2, n_ang, plan.n_det)) * 50)
    i1 = torch.arange(1, n_ang, 4, dtype=torch.int32, device="cuda")
    i2 = torch.arange(0, n_ang, 2, dtype=torch.int32, device="cuda")
    r = torch.empty(2, i1.numel(), plan.n_det, device="cuda")
    p = torch.empty(3, i2.numel(), plan.n_det, device="cuda")
    S.proj_fwd_multi(plan, [S.Job(x1, r, i1, aux=y), S.Job(x2, p, i2)])
    assert torch.equal(r, S.proj_fwd(plan, x1, i1, y=y))
    ref = S.proj_fwd(plan, x2.float(), i2)
    assert torch.allclose(p, ref, rtol=0, atol=1e-4 * float(ref.abs().max()))
    g1 = torch.empty(2, N, N, device="cuda")
    add = dev(rng.random((3, N, N)))
    g2 = torch.empty(3, N, N, device="cuda")
    S.proj_adj_multi(plan, [S.Job(r, g1, i1, alpha=-0.25), S.Job(p, g2, i2, aux=add, beta=1.0)])
    assert torch.equal(g1, S.proj_adj(plan, r, i1, alpha=-0.25))
    ref2 = S.proj_adj(plan, p, i2) + add
    assert rel(host(g2), host(ref2)) <= FP32_TOL


def test_operators_are_deterministic(S):
    """Every kernel fixes its summation order: two runs agree bit for bit."""
    N, n_ang = 128, 36
    plan = S.Plan(N, n_ang)
    rng = np.random.default_rng(9)
    x = dev(rng.standard_normal((2, N, N)))
    p = dev(rng.standard_normal((2, n_ang, plan.n_det)))
    for fn, arg in ((S.proj_fwd, x), (S.proj_adj, p), (S.backproject, p),
                    (S.backproject_adj, x), (S.fbp, p), (S.fbp_adj, x)):
        assert torch.equal(fn(plan, arg), fn(plan, arg))


@pytest.mark.parametrize("N,n_ang,B,m", [(64, 60, 2, 15), (100, 30, 1, 30), (37, 24, 3, 8)])
def test_adjoint_jobs_sharing_the_sketch_match_single_calls(S, N, n_ang, B, m):
    """Two A^T jobs over the same angle list with 4 images of the second per
    image of the first run as one launch in which each CTA carries one image
    of the first job along its group of 4: the results must be bitwise those
    of separate calls, and match the oracle."""
    plan = S.Plan(N, n_ang)
    idx_np = _idx(n_ang, m, 5)
    idx = None if idx_np is None else torch.tensor(idx_np, dtype=torch.int32, device="cuda")
    gen = torch.Generator().manual_seed(N)
    r = torch.randn((B, m, plan.n_det), generator=gen).cuda()
    v = torch.randn((4 * B, m, plan.n_det), generator=gen).cuda()
    aux = torch.randn((4 * B, N, N), generator=gen).cuda()
    o0 = torch.empty((B, N, N), device="cuda")
    o1 = torch.empty((4 * B, N, N), device="cuda")
    S.proj_adj_multi(plan, [S.Job(r, o0, idx, alpha=-0.5), S.Job(v, o1, idx, aux=aux, beta=1.0)])
    ref0 = S.proj_adj(plan, r, idx, alpha=-0.5)
    ref1 = S.proj_adj(plan, v, idx, alpha=1.0, beta=1.0, out=aux.clone())
    torch.cuda.synchronize()
    assert torch.equal(o0, ref0)
    assert torch.equal(o1, ref1)
    ang = plan.angles_deg if idx_np is None else O.select(plan.angles_deg, idx_np)
    assert rel(host(o0), -0.5 * O.proj_adj(host(r), ang, N)) <= FP32_TOL
    assert rel(host(o1), O.proj_adj(host(v), ang, N) + host(aux)) <= FP32_TOL


@pytest.mark.parametrize("N,rows", [(20, 7), (64, 60), (100, 31), (256, 180), (512, 120),
                                    (1000, 5)])
def test_filter_fft_matches_oracle(S, N, rows):
    """The FFT form of H: the same linear convolution (zero padding to a power
    of two >= 2 n_det - 1), odd and even row counts, short rows (direct form)."""
    plan = S.Plan(N, 4)
    rng = np.random.default_rng(N + rows)
    p = rng.standard_normal((rows, plan.n_det))
    got = S.filter_fft(plan, dev(p), 0.5)
    assert rel(host(got), 0.5 * O.ramlak(p)) <= FP32_TOL
    pb = dev(p).to(torch.bfloat16)
    gb = S.filter_fft(plan, pb, 0.5)
    assert gb.dtype == torch.bfloat16
    assert rel(host(gb), 0.5 * O.ramlak(host(pb))) <= 1e-2
    with pytest.raises(RuntimeError):
        x = dev(p)
        S.filter_fft(plan, x, 1.0, out=x)


@pytest.mark.parametrize("N,rows", [(5, 3), (20, 7), (64, 60), (100, 31), (256, 180), (512, 120),
                                    (1024, 17), (1500, 5)])
def test_filter_tc_matches_oracle(S, N, rows):
    """The tensor-core form of H (TF32 head + tail products): ragged row and
    bin counts around the 16 x 32 tiles, the step's 120 x 725 rows, and rows
    beyond 2048 bins (direct form)."""
    plan = S.Plan(N, 4)
    rng = np.random.default_rng(3 * N + rows)
    p = rng.standard_normal((rows, plan.n_det))
    got = S.filter_tc(plan, dev(p), 0.5)
    ref = 0.5 * O.ramlak(p)
    assert rel(host(got), ref) <= FP32_TOL
    # near the direct form: both are FP32 evaluations of the same sums
    assert rel(host(got), host(S.filter(plan, dev(p), 0.5))) <= 2e-6
    pb = dev(p).to(torch.bfloat16)
    gb = S.filter_tc(plan, pb, 0.5)
    assert gb.dtype == torch.bfloat16
    assert rel(host(gb), 0.5 * O.ramlak(host(pb))) <= 1e-2
    again = S.filter_tc(plan, dev(p), 0.5)
    assert torch.equal(again, got)
    with pytest.raises(RuntimeError):
        x = dev(p)
        S.filter_tc(plan, x, 1.0, out=x)
