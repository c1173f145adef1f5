"""Checkpoint and resume of test-time training (Algorithm 2 with the
residual network F(u) = u + theta): a run saved after k iterations and
resumed in a fresh object continues exactly as the uninterrupted run (the
same draws, losses and theta, bit for bit)."""
import numpy as np
import pytest
import torch

from paper_2411_05771_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def problem():
    from paper_2411_05771_gb300 import skei as S
    N, n_ang = 64, 60
    plan = S.Plan(N, n_ang)
    x_gt = torch.tensor(I.rasterize(I.random_ellipses(0), N)[None], device="cuda",
                        dtype=torch.float32)
    y = S.proj_fwd(plan, x_gt)
    x0 = S.fbp(plan, y)
    return S, plan, x0, y


@pytest.mark.parametrize("dtype,G,m,mc_sketched", [
    (torch.float32, 4, 15, True),    # Algorithm 2's form: MC on the sketch too
    (torch.float32, 3, 20, False),   # MC on all angles, G = 3
    (torch.bfloat16, 4, 15, True),   # BF16 storage
])
def test_resumed_run_continues_bitwise(problem, tmp_path, dtype, G, m, mc_sketched):
    from paper_2411_05771_gb300.ttt import ResidualTTT
    S, plan, x0, y = problem
    x0, y = x0.to(dtype), y.to(dtype)
    cfg = dict(m=m, G=G, mc_sketched=mc_sketched, lam=0.7, lr=1e-3, seed=11)
    full = ResidualTTT(plan, x0, y, **cfg)
    ref = [full.step()[0].item() for _ in range(8)]
    part = ResidualTTT(plan, x0, y, **cfg)
    first = [part.step()[0].item() for _ in range(4)]
    path = tmp_path / "run.pt"
    part.save(path)
    del part
    resumed = ResidualTTT.load(path, plan, x0, y, **cfg)
    assert resumed.t == 4
    rest = [resumed.step()[0].item() for _ in range(4)]
    assert first + rest == ref
    assert torch.equal(resumed.theta, full.theta)
    assert torch.equal(resumed.m1, full.m1) and torch.equal(resumed.v1, full.v1)
    assert np.isfinite(ref).all()
    assert plan.status() == 0


def test_checkpoint_of_another_run_is_refused(problem, tmp_path):
    from paper_2411_05771_gb300.ttt import ResidualTTT
    S, plan, x0, y = problem
    run = ResidualTTT(plan, x0, y, m=15, G=4)
    run.step()
    path = tmp_path / "run.pt"
    run.save(path)
    with pytest.raises(ValueError):
        ResidualTTT.load(path, plan, x0, y, m=20, G=4)
