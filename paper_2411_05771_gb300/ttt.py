"""Test-time training with the residual network F(u) = u + theta
(Algorithm 2: the SkEI loss of Eq. (e:skeilossttt) minimised over theta by
Adam, one measurement at a time), one `skei_ttt_residual_step` per
iteration, with checkpoint and resume.

The operators are stateless, so the state of a run is: theta, Adam's two
moments, the iteration count, and the generator of the per-iteration draws
(the sketch offset S_k and the G rotation angles).  `save` writes it with
torch.save; `ResidualTTT.load` rebuilds a run that continues exactly as the
uninterrupted one would (same draws, same kernels, same bits).
"""
import numpy as np
import torch

from . import inputs as I
from . import skei as S

_FORMAT = "skei-residual-ttt-1"


class ResidualTTT:
    """Algorithm 2 on measurements y [B, n_angles, n_det] from the start
    x0 [B, N, N] (e.g. the FBP of y), both on the GPU, FP32 or BF16 storage.

    m: angles per sketch (divides n_angles; m = n_angles: no sketch);
    mc_sketched: the MC term on the same sketch (Algorithm 2's form, scaled
    by n_angles / m) or on all angles; G rotations per measurement, drawn
    U[0, 360) degrees every iteration with the sketch offset; lam: the
    weight of the EI term; Adam with learning rate lr (betas 0.9, 0.999,
    eps 1e-8); seed: the draws' generator."""

    def __init__(self, plan: S.Plan, x0: torch.Tensor, y: torch.Tensor, m: int, G: int = 4,
                 mc_sketched: bool = True, lam: float = 1.0, lr: float = 5e-4, seed: int = 0):
        if x0.dim() != 3 or y.dim() != 3 or y.shape[0] != x0.shape[0]:
            raise ValueError("x0 must be [B, N, N] and y [B, n_angles, n_det]")
        if m <= 0 or plan.n_angles % m != 0:
            raise ValueError("the sketch size must divide the angle count")
        self.plan, self.x0, self.y = plan, x0, y
        self.B, self.N, self.G, self.m = x0.shape[0], plan.N, G, m
        self.sketched = m < plan.n_angles
        self.mc_sketched = mc_sketched and self.sketched
        self.mc_scale = plan.n_angles / m if self.mc_sketched else 1.0
        self.lam, self.lr = float(lam), float(lr)
        dev = x0.device
        f32 = dict(dtype=torch.float32, device=dev)
        self.theta = torch.zeros((self.N, self.N), **f32)
        self.m1 = torch.zeros_like(self.theta)
        self.v1 = torch.zeros_like(self.theta)
        self.t = 0                                   # iterations done
        self.rng = np.random.default_rng(seed)
        self._step_dev = torch.zeros((), dtype=torch.int32, device=dev)
        self._idx = torch.zeros(m, dtype=torch.int32, device=dev)
        self._g = torch.zeros((self.B, G), dtype=torch.float64, device=dev)
        mc_m = m if self.mc_sketched else plan.n_angles
        code = S.F32 if x0.dtype == torch.float32 else S.BF16
        self._work = torch.empty(S.ttt_residual_workspace_size(plan, code, self.B, G, mc_m, m),
                                 dtype=torch.uint8, device=dev)
        self._out = None

    # ------------------------------------------------------------ steps --
    def _draw(self):
        """The next iteration's sketch S_k and rotations (host generator)."""
        n = self.plan.n_angles
        off = I.random_sketch_offset(self.rng, n, self.m) if self.sketched else 0
        idx = I.sketch_indices(n, self.m, off) if self.sketched else np.arange(n)
        return idx.astype(np.int32), I.rotation_angles(self.rng, self.B, self.G)

    def step(self):
        """One iteration; returns (loss, mc, ei) as device tensors (FP64)."""
        idx, g = self._draw()
        self.t += 1
        self._idx.copy_(torch.as_tensor(idx))
        self._g.copy_(torch.as_tensor(g))
        self._step_dev.fill_(self.t)
        sk = self._idx if self.sketched else None
        mc = sk if self.mc_sketched else None
        self._out = S.ttt_residual_step(self.plan, self.x0, self.theta, self.m1, self.v1,
                                        self._step_dev, self.y, self._g, mc, sk, self.lam,
                                        self.mc_scale, self.lr, out=self._out, work=self._work)
        return self._out[8], self._out[9], self._out[10]

    def output(self) -> torch.Tensor:
        """The current reconstruction F(x0) = x0 + theta (FP32)."""
        return self.x0.float() + self.theta

    # ---------------------------------------------- checkpoint / resume --
    def _config(self) -> dict:
        return {"B": self.B, "N": self.N, "G": self.G, "m": self.m,
                "mc_sketched": self.mc_sketched, "lam": self.lam, "lr": self.lr,
                "n_angles": self.plan.n_angles, "n_det": self.plan.n_det}

    def state_dict(self) -> dict:
        return {"format": _FORMAT, "t": self.t, "theta": self.theta.detach().cpu(),
                "m": self.m1.detach().cpu(), "v": self.v1.detach().cpu(),
                "rng": self.rng.bit_generator.state, "config": self._config()}

    def load_state_dict(self, sd: dict) -> None:
        if sd.get("format") != _FORMAT:
            raise ValueError("not a residual-TTT checkpoint")
        mine = self._config()
        if sd["config"] != mine:
            raise ValueError(f"checkpoint of another run: {sd['config']} vs {mine}")
        self.theta.copy_(sd["theta"])
        self.m1.copy_(sd["m"])
        self.v1.copy_(sd["v"])
        self.t = int(sd["t"])
        self.rng.bit_generator.state = sd["rng"]

    def save(self, path) -> None:
        torch.save(self.state_dict(), path)

    @classmethod
    def load(cls, path, plan: S.Plan, x0: torch.Tensor, y: torch.Tensor, **config):
        """A run with the given problem and configuration (as passed to the
        constructor) resumed from the checkpoint at `path`."""
        run = cls(plan, x0, y, **config)
        run.load_state_dict(torch.load(path, weights_only=True))   # tensors and plain values only
        return run
