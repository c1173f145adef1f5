"""GPU parity of the batched persistent schedule (skei_batch_*): one operator
over many instances with different image sizes, angle lists, sketches and
storage types, in one persistent launch per kernel.

Each item is checked two ways: bitwise against the single-instance entry
point on the same item (the schedule must not change any result), and
against the FP64 oracle (rel-L2 <= 1e-5 for FP32 storage, <= 1e-2 for BF16
storage against the oracle on the same BF16-rounded input)."""
import numpy as np
import pytest
import torch

import oracle as O
from paper_2411_05771_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5
BF16_TOL = 1e-2


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


# (N, n_angles, B, m, storage): ragged sizes, full and sketched angle sets,
# both storage types; the last item shares the first item's plan with
# another sketch
MIXED = [(64, 60, 2, 15, torch.float32), (48, 36, 1, 36, torch.float32),
         (37, 24, 3, 8, torch.bfloat16), (100, 30, 1, 10, torch.float32),
         (64, 90, 1, 45, torch.bfloat16), (33, 20, 2, 5, torch.float32),
         (64, 60, 1, 30, torch.float32)]


def _sketch(n_ang, m, seed):
    if m == n_ang:
        return None
    off = I.random_sketch_offset(np.random.default_rng(seed), n_ang, m)
    return I.sketch_indices(n_ang, m, off)


def _items(S, op, spec, seed=0, scales=None):
    """Plans, sketches, inputs and outputs of the batch items."""
    gen = torch.Generator().manual_seed(seed)
    plans, out = {}, []
    for q, (N, n_ang, B, m, dt) in enumerate(spec):
        key = (N, n_ang)
        if key not in plans:
            plans[key] = S.Plan(N, n_ang)
        plan = plans[key]
        idx_np = _sketch(n_ang, m, seed * 100 + q)
        idx = None if idx_np is None else torch.tensor(idx_np, dtype=torch.int32, device="cuda")
        img, sino = (B, N, N), (B, m, plan.n_det)
        shp_in, shp_out = {S.PROJ_FWD: (img, sino), S.PROJ_ADJ: (sino, img),
                           S.BACKPROJECT: (sino, img), S.BACKPROJECT_ADJ: (img, sino),
                           S.FILTER: (sino, sino), S.FBP: (sino, img)}[op]
        inp = torch.randn(shp_in, generator=gen).to(dt).cuda()
        outp = torch.full(shp_out, float("nan"), dtype=dt, device="cuda")
        scale = 1.0 if scales is None else scales[q]
        out.append(dict(plan=plan, idx=idx, idx_np=idx_np, inp=inp, out=outp, scale=scale,
                        m=m, dt=dt))
    return out


def _single(S, op, it):
    """The single-instance entry point on one item."""
    p, idx, x, a = it["plan"], it["idx"], it["inp"], it["scale"]
    if op == S.PROJ_FWD:
        y = S.proj_fwd(p, x, idx)
        return y if a == 1.0 else y * a   # a power of two in the tests: exact
    if op == S.PROJ_ADJ:
        return S.proj_adj(p, x, idx, alpha=a)
    if op == S.BACKPROJECT:
        return S.backproject(p, x, idx, alpha=a)
    if op == S.BACKPROJECT_ADJ:
        return S.backproject_adj(p, x, idx, alpha=a)
    if op == S.FILTER:
        return S.filter(p, x, a)
    y = S.fbp(p, x, idx)
    return y if a == 1.0 else y * a


def _oracle(S, op, it):
    p = it["plan"]
    ang = p.angles_deg if it["idx_np"] is None else O.select(p.angles_deg, it["idx_np"])
    x = host(it["inp"])  # the stored (possibly BF16-rounded) input
    a = it["scale"]
    if op == S.PROJ_FWD:
        return a * O.proj_fwd(x, ang, p.n_det)
    if op == S.PROJ_ADJ:
        return a * O.proj_adj(x, ang, p.N)
    if op == S.BACKPROJECT:
        return a * O.backproject(x, ang, p.N)
    if op == S.BACKPROJECT_ADJ:
        return a * O.backproject_adj(x, ang, p.n_det)
    if op == S.FILTER:
        return a * O.ramlak(x)
    return a * O.fbp(x, ang, p.N)


OPS = ["PROJ_FWD", "PROJ_ADJ", "BACKPROJECT", "BACKPROJECT_ADJ", "FILTER", "FBP"]


@pytest.mark.parametrize("opname", OPS)
def test_batch_matches_single_calls_and_oracle(S, opname):
    op = getattr(S, opname)
    scales = [1.0, 0.5, 1.0, 2.0, 1.0, 0.25, 1.0]
    items = _items(S, op, MIXED, seed=1, scales=scales)
    batch = S.Batch(op, [S.BatchItem(it["plan"], it["inp"], it["out"], it["idx"], it["scale"])
                         for it in items])
    batch.run()
    torch.cuda.synchronize()
    for q, it in enumerate(items):
        got = it["out"]
        assert torch.isfinite(got.float()).all(), f"item {q}: output not fully written"
        ref = _single(S, op, it)
        assert torch.equal(got, ref), f"item {q}: batch differs from the single-instance call"
        tol = FP32_TOL if it["dt"] == torch.float32 else BF16_TOL
        assert rel(host(got), _oracle(S, op, it)) <= tol, f"item {q} vs oracle"


def test_batch_rerun_graph_replay_and_tune(S):
    """The work queue resets itself: runs in a row, replays of a captured
    graph, and every shape the tuner tries give the same bits."""
    items = _items(S, S.PROJ_FWD, MIXED, seed=2)
    batch = S.Batch(S.PROJ_FWD, [S.BatchItem(it["plan"], it["inp"], it["out"], it["idx"])
                                 for it in items])
    batch.run()
    first = [it["out"].clone() for it in items]
    for _ in range(3):
        for it in items:
            it["out"].fill_(float("nan"))
        batch.run()
        for it, f in zip(items, first):
            assert torch.equal(it["out"], f)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        batch.run()  # warm outside the capture
        st.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=st):
            batch.run()
        for _ in range(3):
            for it in items:
                it["out"].fill_(float("nan"))
            g.replay()
        st.synchronize()
    for it, f in zip(items, first):
        assert torch.equal(it["out"], f)
    # new inputs written into the baked buffers are picked up by a replay
    items[0]["inp"].mul_(2.0)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(items[0]["out"], 2.0 * first[0])
    items[0]["inp"].mul_(0.5)
    batch.tune(reps=2)
    info = batch.info(0)
    assert info["phases"] == 1 and 1 <= info["block"] <= 8 and info["tasks"] > 0
    for it in items:
        it["out"].fill_(float("nan"))
    batch.run()
    torch.cuda.synchronize()
    for it, f in zip(items, first):
        assert torch.equal(it["out"], f)


def test_batch_fbp_tune_keeps_results(S):
    items = _items(S, S.FBP, MIXED, seed=3)
    batch = S.Batch(S.FBP, [S.BatchItem(it["plan"], it["inp"], it["out"], it["idx"])
                            for it in items])
    batch.tune(reps=1)
    assert batch.info(0)["phases"] == 2
    batch.run()
    torch.cuda.synchronize()
    for it in items:
        assert torch.equal(it["out"], _single(S, S.FBP, it))


def test_batch_tune_cache_on_disk(S, tmp_path, monkeypatch):
    """SKEI_AUTOTUNE_CACHE: a tuned batch records its phases' shapes; a new
    batch of the same items takes them from the file without timing (shown
    by a recorded shape the timing would not pick), and keeps its results."""
    path = tmp_path / "tune.txt"
    monkeypatch.setenv("SKEI_AUTOTUNE_CACHE", str(path))
    items = _items(S, S.FBP, MIXED, seed=4)
    mk = lambda: S.Batch(S.FBP, [S.BatchItem(it["plan"], it["inp"], it["out"], it["idx"])  # noqa: E731
                                 for it in items])
    first = mk()
    first.tune(reps=1)
    lines = path.read_text().splitlines()
    assert len(lines) == 2                      # the filter and the back-projection phases
    assert all("\t" in ln and ln.split("\t")[1].isdigit() for ln in lines)
    # overwrite the recorded shapes with 1 (a valid candidate of every phase)
    path.write_text("".join(ln.rsplit("\t", 1)[0] + "\t1\n" for ln in lines))
    second = mk()
    second.tune(reps=1)
    assert [second.info(q)["block"] for q in range(2)] == [1, 1]
    assert path.read_text().count("\n") == 2   # nothing timed, nothing appended
    second.run()
    torch.cuda.synchronize()
    for it in items:
        assert torch.equal(it["out"], _single(S, S.FBP, it))
    # another item set is not in the file: timed and appended
    other = _items(S, S.FBP, MIXED[:3], seed=5)
    third = S.Batch(S.FBP, [S.BatchItem(it["plan"], it["inp"], it["out"], it["idx"])
                            for it in other])
    third.tune(reps=1)
    assert path.read_text().count("\n") == 4


def test_batch_rejects_bad_items(S):
    p = S.Plan(32, 12)
    x = torch.zeros(1, 32, 32, device="cuda")
    y = torch.zeros(1, 12, p.n_det + 1, device="cuda")
    with pytest.raises(ValueError):
        S.Batch(S.PROJ_FWD, [S.BatchItem(p, x, y)])
    with pytest.raises(TypeError):
        S.Batch(S.PROJ_FWD, [S.BatchItem(p, x.cpu(), y[..., :-1].contiguous())])
    idx = torch.tensor([0, 13], dtype=torch.int32, device="cuda")   # 13 >= n_angles
    out = torch.zeros(1, 2, p.n_det, device="cuda")
    b = S.Batch(S.PROJ_FWD, [S.BatchItem(p, x, out, idx)])
    p.status(reset=True)
    b.run()
    torch.cuda.synchronize()
    assert p.status() & 1                   # the bad row was reported
    assert bool((out[0, 1] == 0).all())     # and zeroed, not read


def _config4(S, dt, seed=4):
    """16 instances mixing 256^2 (360 angles, 363 bins) and 512^2 (720
    angles, 725 bins), sketch sizes drawn from {45, 90, 180, 360}."""
    rng = np.random.default_rng(seed)
    sizes = [(256, 360), (512, 720)] * 8
    ms = rng.choice([45, 90, 180, 360], size=16)
    return [(N, n, 1, int(m), dt) for (N, n), m in zip(sizes, ms)]


@pytest.mark.parametrize("dt", [torch.float32, torch.bfloat16])
def test_batch_mixed_256_512_full_size(S, dt):
    spec = _config4(S, dt)
    for op in (S.PROJ_FWD, S.PROJ_ADJ, S.FBP):
        items = _items(S, op, spec, seed=5)
        batch = S.Batch(op, [S.BatchItem(it["plan"], it["inp"], it["out"], it["idx"])
                             for it in items])
        batch.run()
        torch.cuda.synchronize()
        for q, it in enumerate(items):
            assert torch.equal(it["out"], _single(S, op, it)), f"op {op} item {q}"
        # the oracle on the first 256^2 and the first 512^2 instance; for A
        # three sampled angles of each sketch, the adjoint and FBP in full
        for q in (0, 1):
            it = items[q]
            p = it["plan"]
            ang = p.angles_deg if it["idx_np"] is None else O.select(p.angles_deg, it["idx_np"])
            tol = FP32_TOL if dt == torch.float32 else BF16_TOL
            if op == S.PROJ_FWD:
                rows = [0, it["m"] // 2, it["m"] - 1]
                ref = O.proj_fwd(host(it["inp"]), ang[rows], p.n_det)
                assert rel(host(it["out"][:, rows]), ref) <= tol
            else:
                assert rel(host(it["out"]), _oracle(S, op, it)) <= tol
