"""skei_fbp_noalloc: the FBP entry point for callers that cannot allocate
device memory (a pool owns it all, a real-time loop forbids allocation, a
plugin host gives no allocator).  It must give what skei_fbp gives, call
after call, although every call reuses the same static scratch array inside
the library, and it must refuse sizes beyond that array.

This file is collected last on purpose: it also has to pass when it runs
alone in a fresh process, where its first call does the one-time lookup of
the scratch array's device address."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu
FP32_TOL = 1e-5
BF16_TOL = 1e-2


@pytest.fixture(scope="module")
def S():
    from paper_2411_05771_gb300 import skei
    return skei


def _rel(a, b):
    a, b = a.double(), b.double()
    return float((a - b).norm() / b.norm())


def test_noalloc_fbp_matches_fbp_on_two_calls_in_a_row(S):
    torch.manual_seed(0)
    N, n_ang, m, B = 64, 60, 15, 2
    plan = S.Plan(N, n_ang)
    idx = torch.arange(3, n_ang, n_ang // m, dtype=torch.int32, device="cuda")
    # two different inputs, so a stale scratch from the first call would show
    sinos = [torch.randn(B, m, plan.n_det, device="cuda") for _ in range(2)]
    outs = [torch.empty(B, N, N, device="cuda") for _ in range(2)]
    for sino, out in zip(sinos, outs):
        S.fbp_noalloc(plan, sino, idx, out=out)       # the C ABI, no allocation
    torch.cuda.synchronize()
    for sino, out in zip(sinos, outs):
        ref = S.fbp(plan, sino, idx)
        assert _rel(out, ref) <= FP32_TOL
    # full angle set, BF16 storage, again twice in a row
    full = torch.randn(1, n_ang, plan.n_det, device="cuda").to(torch.bfloat16)
    ref = S.fbp(plan, full)
    for _ in range(2):
        got = S.fbp_noalloc(plan, full)
        assert _rel(got.float(), ref.float()) <= BF16_TOL


def test_noalloc_fbp_rejects_sizes_beyond_its_scratch(S):
    N, n_ang = 512, 720
    plan = S.Plan(N, n_ang)
    B = S.FBP_NOALLOC_MAX_FLOATS // (n_ang * plan.n_det) + 1
    sino = torch.zeros(B, n_ang, plan.n_det, device="cuda")
    out = torch.full((B, N, N), 7.0, device="cuda")
    with pytest.raises(RuntimeError, match="static scratch"):
        S.fbp_noalloc(plan, sino, out=out)
    torch.cuda.synchronize()
    assert bool((out == 7.0).all())   # nothing was launched
    # the largest batch that fits still works (B m n_det <= the maximum:
    # the size check is pinned from both sides)
    B_max = S.FBP_NOALLOC_MAX_FLOATS // (n_ang * plan.n_det)
    ok = torch.randn(B_max, n_ang, plan.n_det, device="cuda")
    assert _rel(S.fbp_noalloc(plan, ok), S.fbp(plan, ok)) <= FP32_TOL
