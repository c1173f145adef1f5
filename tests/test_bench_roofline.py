"""The bench's roofline arithmetic on the host (no GPU): the work counts it
divides by and the choice of the binding roof."""
import os
import sys
from types import SimpleNamespace

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _plan(N, n_det, angles):
    return SimpleNamespace(N=N, n_det=n_det, angles_deg=np.asarray(angles, dtype=np.float64))


def test_joseph_crossings_at_axis_angles():
    # N = 8, 13 bins: at 0 and 90 degrees the rays sit at positions
    # -2.5 .. 9.5 on every line, 9 of them inside (-1, 8), on each of 8 lines
    p = _plan(8, 13, [0.0, 90.0])
    assert bench.joseph_samples(p, 1, [0]) == 72
    assert bench.joseph_samples(p, 1, [1]) == 72
    assert bench.joseph_samples(p, 3, [0, 1]) == 3 * 144


def test_joseph_crossings_of_a_diagonal_cover_the_image_once_per_line():
    # every line of the image is crossed by the rays of an angle whose
    # spacing along the line is |1/cos|: about N |cos| rays per line
    N = 64
    p = _plan(N, int(np.ceil(N * np.sqrt(2))) | 1, [30.0])
    n = bench.joseph_samples(p, 1, [0])
    assert abs(n / N - N * np.cos(np.radians(30.0))) <= 2.0


def _arm(N, views, m, G, B, mc_sketched=True):
    wl = bench.Workload(N=N, views=views, m=m, G=G, B=B, mc_sketched=mc_sketched)
    idx = np.arange(0, views, views // m)
    torch = pytest.importorskip("torch")
    return SimpleNamespace(wl=wl, idx=torch.tensor(idx), m=m, mc_m=wl.mc_m,
                           sketched=wl.sketched)


def test_roofline_picks_the_binding_roof():
    N, views, m = 64, 60, 15
    plan = _plan(N, 91, 180.0 * np.arange(views) / views)
    arm = _arm(N, views, m, 4, 1)
    roofs = {"fp32_flops": 80e12, "smem_bytes": 40e12, "dram_read_bytes": 7e12}
    peaks = {"hbm_gbs": 6800.0}
    t_us = 10.0
    e = bench.roofline_entry(plan, arm, {"backproject_adj": t_us}, "backproject_adj", roofs,
                             peaks)
    samples = bench.pixel_angles(plan, 4, m)
    t_fp32 = 7 * samples / 80e12
    t_smem = 8 * samples / 40e12
    assert e["bound"] == "smem"          # 8 B / 40 TB/s beats 7 flop / 80 TF/s
    assert e["frac"] == pytest.approx(t_smem / (t_us * 1e-6))
    assert e["frac_by_roof"]["fp32"] == pytest.approx(t_fp32 / (t_us * 1e-6), abs=1e-4)  # 4 decimals
    assert e["achieved"] == pytest.approx(8 * samples / (t_us * 1e-6) / 1e9)
    assert e["peak"] == pytest.approx(40e3)
