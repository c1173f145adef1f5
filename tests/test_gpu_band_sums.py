"""GPU parity of the workspace forms of the line-summing operators
(skei_proj_fwd_multi_ws: Joseph A; skei_backproject_adj_multi_ws: B^T):
per-band sums in a workspace, then an ordered reduction.  Checked against
the FP64 oracle (rel-L2 <= 1e-5; BF16 storage <= 1e-2 on the same rounded
input) and against the forms without workspace (same operator, different
summation order: rel-L2 <= 1e-6)."""
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


def host(t):
    return t.detach().double().cpu().numpy()


def _sk(n_ang, m, seed):
    if m == n_ang:
        return None
    off = I.random_sketch_offset(np.random.default_rng(seed), n_ang, m)
    return I.sketch_indices(n_ang, m, off)


# (N, n_angles, (B, m) of job 0, (B, m) of job 1): single images and groups
# of 4 with a remainder, ragged N, full and sketched angle sets
CASES = [(64, 60, (1, 60), (4, 15)), (37, 24, (3, 8), (5, 24)), (100, 30, (8, 10), (1, 30)),
         (256, 180, (1, 180), (8, 45)), (512, 60, (1, 30), (4, 30))]


@pytest.mark.parametrize("N,n_ang,j0,j1", CASES)
def test_forward_with_band_sums(S, N, n_ang, j0, j1):
    plan = S.Plan(N, n_ang)
    gen = torch.Generator().manual_seed(N + n_ang)
    jobs, refs = [], []
    for q, (B, m) in enumerate((j0, j1)):
        idx_np = _sk(n_ang, m, q)
        idx = None if idx_np is None else torch.tensor(idx_np, dtype=torch.int32, device="cuda")
        x = torch.randn((B, N, N), generator=gen).cuda()
        out = torch.full((B, m, plan.n_det), float("nan"), device="cuda")
        ang = plan.angles_deg if idx_np is None else O.select(plan.angles_deg, idx_np)
        if q == 0:   # residual form on the first job
            y = torch.randn((B, n_ang, plan.n_det), generator=gen).cuda()
            jobs.append(S.Job(x, out, idx, aux=y))
            yS = host(y) if idx_np is None else host(y)[:, idx_np]
            refs.append(yS - O.proj_fwd(host(x), ang, plan.n_det))
        else:
            jobs.append(S.Job(x, out, idx))
            refs.append(O.proj_fwd(host(x), ang, plan.n_det))
    S.proj_fwd_multi_ws(plan, jobs)
    torch.cuda.synchronize()
    for q, (jb, ref) in enumerate(zip(jobs, refs)):
        assert torch.isfinite(jb.out).all(), f"job {q}: output not fully written"
        assert rel(host(jb.out), ref) <= FP32_TOL, f"job {q} vs oracle"
    # agrees with the form without workspace
    outs = [jb.out.clone() for jb in jobs]
    S.proj_fwd_multi(plan, jobs)
    for q, (jb, o) in enumerate(zip(jobs, outs)):
        assert rel(host(o), host(jb.out)) <= 1e-6, f"job {q} vs cluster form"


@pytest.mark.parametrize("N,n_ang,B,m", [(37, 24, 1, 8), (64, 60, 3, 15), (256, 180, 2, 45),
                                         (512, 60, 1, 60),
                                         # N % 8 = 4: the riding image's general staging
                                         (100, 36, 2, 12),
                                         # N > 512: staged after the group, not prefetched
                                         (520, 36, 1, 12)])
def test_forward_band_sums_single_image_rides_with_its_group(S, N, n_ang, B, m):
    """Two jobs on one angle list with 4 images of job 1 per image of job 0
    (the MC and EI terms of a step with G = 4): image b of job 0 is summed in
    the CTAs of job 1's images 4b .. 4b+3.  Its sums are those of the same
    launch with the list given twice (no riding), bit for bit."""
    plan = S.Plan(N, n_ang)
    gen = torch.Generator().manual_seed(3 * N + m)
    idx_np = _sk(n_ang, m, 5)
    idx = None if idx_np is None else torch.tensor(idx_np, dtype=torch.int32, device="cuda")
    x0 = torch.randn((B, N, N), generator=gen).cuda()
    x1 = torch.randn((4 * B, N, N), generator=gen).cuda()
    y = torch.randn((B, n_ang, plan.n_det), generator=gen).cuda()
    nan = dict(fill_value=float("nan"), device="cuda")
    jobs = [S.Job(x0, torch.full((B, m, plan.n_det), **nan), idx, aux=y),
            S.Job(x1, torch.full((4 * B, m, plan.n_det), **nan), idx)]
    S.proj_fwd_multi_ws(plan, jobs)
    idx2 = None if idx is None else idx.clone()
    if idx2 is None:   # a full list given explicitly: same angles, another pointer
        idx2 = torch.arange(n_ang, dtype=torch.int32, device="cuda")
    apart = [S.Job(x0, torch.full((B, m, plan.n_det), **nan), idx2, aux=y),
             S.Job(x1, torch.full((4 * B, m, plan.n_det), **nan), idx)]
    S.proj_fwd_multi_ws(plan, apart)
    torch.cuda.synchronize()
    ang = plan.angles_deg if idx_np is None else O.select(plan.angles_deg, idx_np)
    yS = host(y) if idx_np is None else host(y)[:, idx_np]
    assert rel(host(jobs[0].out), yS - O.proj_fwd(host(x0), ang, plan.n_det)) <= FP32_TOL
    assert rel(host(jobs[1].out), O.proj_fwd(host(x1), ang, plan.n_det)) <= FP32_TOL
    assert torch.equal(jobs[0].out, apart[0].out)
    assert torch.equal(jobs[1].out, apart[1].out)


@pytest.mark.parametrize("N,n_ang,j0,j1", CASES)
def test_backproject_transpose_with_band_sums(S, N, n_ang, j0, j1):
    plan = S.Plan(N, n_ang)
    gen = torch.Generator().manual_seed(7 * N + n_ang)
    jobs, refs = [], []
    for q, (B, m) in enumerate((j0, j1)):
        idx_np = _sk(n_ang, m, q + 2)
        idx = None if idx_np is None else torch.tensor(idx_np, dtype=torch.int32, device="cuda")
        x = torch.randn((B, N, N), generator=gen).cuda()
        out = torch.full((B, m, plan.n_det), float("nan"), device="cuda")
        ang = plan.angles_deg if idx_np is None else O.select(plan.angles_deg, idx_np)
        alpha = 0.5 if q else 1.0
        jobs.append(S.Job(x, out, idx, alpha=alpha))
        refs.append(alpha * O.backproject_adj(host(x), ang, plan.n_det))
    S.backproject_adj_multi_ws(plan, jobs)
    torch.cuda.synchronize()
    for q, (jb, ref) in enumerate(zip(jobs, refs)):
        assert torch.isfinite(jb.out).all(), f"job {q}: output not fully written"
        assert rel(host(jb.out), ref) <= FP32_TOL, f"job {q} vs oracle"
        single = S.backproject_adj(plan, jb.inp, jb.idx, alpha=jb.alpha)
        assert rel(host(jb.out), host(single)) <= 1e-6, f"job {q} vs cluster form"


def test_band_sums_bf16_storage(S):
    N, n_ang = 64, 45
    plan = S.Plan(N, n_ang)
    x = torch.randn((4, N, N)).to(torch.bfloat16).cuda()
    out = torch.empty((4, n_ang, plan.n_det), dtype=torch.bfloat16, device="cuda")
    S.proj_fwd_multi_ws(plan, [S.Job(x, out)])
    ref = O.proj_fwd(host(x), plan.angles_deg, plan.n_det)
    assert rel(host(out), ref) <= 1e-2
    S.backproject_adj_multi_ws(plan, [S.Job(x, out)])
    ref = O.backproject_adj(host(x), plan.angles_deg, plan.n_det)
    assert rel(host(out), ref) <= 1e-2


def test_band_sums_workspace_checks_and_bad_index(S):
    N, n_ang = 32, 12
    plan = S.Plan(N, n_ang)
    x = torch.randn((1, N, N), device="cuda")
    idx = torch.tensor([0, 13], dtype=torch.int32, device="cuda")    # 13 >= n_angles
    out = torch.full((1, 2, plan.n_det), 5.0, device="cuda")
    jobs = [S.Job(x, out, idx)]
    need = S.band_sums_workspace_size(plan, jobs)
    assert need > 0
    small = torch.empty(need - 16, dtype=torch.uint8, device="cuda")
    with pytest.raises(ValueError):
        S.proj_fwd_multi_ws(plan, jobs, work=small)
    plan.status(reset=True)
    S.proj_fwd_multi_ws(plan, jobs)
    torch.cuda.synchronize()
    assert plan.status() & 1                      # the bad row was reported
    assert bool((out[0, 1] == 0).all())           # and zeroed, not read
    ref = O.proj_fwd(host(x), plan.angles_deg[:1], plan.n_det)
    assert rel(host(out[:, :1]), ref) <= FP32_TOL
