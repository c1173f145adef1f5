"""The checkpoint of the test-time training loop holds only tensors and plain
values (it loads with torch.load(weights_only=True)), and the draws'
generator state it stores continues the same sequence (no GPU needed)."""
import numpy as np
import torch


def test_generator_state_round_trip(tmp_path):
    rng = np.random.default_rng(5)
    rng.uniform(size=7)
    sd = {"format": "skei-residual-ttt-1", "t": 3, "theta": torch.arange(4.0),
          "rng": rng.bit_generator.state, "config": {"B": 1, "lam": 0.7, "mc_sketched": True}}
    path = tmp_path / "ck.pt"
    torch.save(sd, path)
    back = torch.load(path, weights_only=True)
    ahead = rng.uniform(size=5)
    resumed = np.random.default_rng(0)
    resumed.bit_generator.state = back["rng"]
    assert np.array_equal(resumed.uniform(size=5), ahead)
    assert torch.equal(back["theta"], sd["theta"]) and back["config"] == sd["config"]
