"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module holds no arithmetic of the method itself (no discrete projector,
filter, back-projector, rotation or loss).  It only draws and rasterises the
test objects that stand in for the CT100 images of the paper (Sec. 4.1.1:
512x512 CT images, 100-view parallel-beam sinograms), and the random choices
the method makes per iteration (Algorithm 2: one sketch S_k and one transform
T_i per iteration), so that both sides of a parity test receive identical
inputs.

Conventions (pixel units, shared by every consumer):
  * image pixel (i, j), i = row from the top, centre
    x_j = j - (N-1)/2, y_i = (N-1)/2 - i  (y points up);
  * the physical field of view is [-1, 1]^2, so physical = pixel * 2/N;
  * detector bin k sits at u_k = k - (n_det-1)/2 (unit spacing);
  * projection angle theta (degrees) has ray normal (cos theta, sin theta),
    and a ray is the line x cos theta + y sin theta = u.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

__all__ = [
    "Ellipses",
    "random_ellipses",
    "rasterize",
    "analytic_sinogram",
    "disk_sinogram",
    "noisy_sinogram",
    "uniform_angles",
    "sketch_indices",
    "random_sketch_offset",
    "rotation_angles",
    "step_rng",
]


@dataclass(frozen=True)
class Ellipses:
    """A sum of constant-intensity ellipses in physical coordinates [-1,1]^2."""

    cx: np.ndarray
    cy: np.ndarray
    a: np.ndarray      # semi-axis along the direction phi
    b: np.ndarray      # semi-axis across it
    phi_deg: np.ndarray
    rho: np.ndarray    # intensity (added where ellipses overlap)


def random_ellipses(seed: int, count: int = 10) -> Ellipses:
    """Ten random ellipses: centres U[-0.8,0.8]^2, semi-axes U(0.05,0.4),
    intensities U(0,1), orientation U[0,180) degrees."""
    rng = np.random.default_rng(seed)
    cx = rng.uniform(-0.8, 0.8, count)
    cy = rng.uniform(-0.8, 0.8, count)
    a = rng.uniform(0.05, 0.4, count)
    b = rng.uniform(0.05, 0.4, count)
    phi = rng.uniform(0.0, 180.0, count)
    rho = rng.uniform(0.0, 1.0, count)
    return Ellipses(cx, cy, a, b, phi, rho)


def rasterize(e: Ellipses, N: int, supersample: int = 1) -> np.ndarray:
    """Point-sample the phantom at pixel centres (optionally s x s sub-samples
    averaged).  Returns float64 [N, N], row 0 at the top."""
    s = int(supersample)
    offs = (np.arange(s) + 0.5) / s - 0.5
    idx = np.arange(N, dtype=np.float64)
    img = np.zeros((N, N), dtype=np.float64)
    for oy in offs:
        for ox in offs:
            X = (idx[None, :] - (N - 1) / 2.0 + ox) * (2.0 / N)
            Y = ((N - 1) / 2.0 - idx[:, None] - oy) * (2.0 / N)
            for cx, cy, a, b, phi, rho in zip(e.cx, e.cy, e.a, e.b, e.phi_deg, e.rho):
                cp, sp = math.cos(math.radians(phi)), math.sin(math.radians(phi))
                dx, dy = X - cx, Y - cy
                xr = dx * cp + dy * sp
                yr = -dx * sp + dy * cp
                img += rho * ((xr / a) ** 2 + (yr / b) ** 2 <= 1.0)
    return img / (s * s)


def analytic_sinogram(e: Ellipses, N: int, angles_deg, n_det: int) -> np.ndarray:
    """Exact line integrals of the continuous phantom along the rays of the
    detector grid, in pixel units (physical value times N/2).

    For one ellipse the chord length through it at normal angle theta and
    offset s' from the centre is 2ab*sqrt(q - s'^2)/q with
    q = a^2 cos^2(theta-phi) + b^2 sin^2(theta-phi) (zero when s'^2 > q).
    Returns float64 [n_angles, n_det]."""
    th = np.radians(np.asarray(angles_deg, dtype=np.float64))[:, None]
    u = (np.arange(n_det, dtype=np.float64) - (n_det - 1) / 2.0)[None, :]
    S = u * (2.0 / N)
    out = np.zeros((th.shape[0], n_det), dtype=np.float64)
    for cx, cy, a, b, phi, rho in zip(e.cx, e.cy, e.a, e.b, e.phi_deg, e.rho):
        sp = S - (cx * np.cos(th) + cy * np.sin(th))
        d = th - math.radians(phi)
        q = (a * np.cos(d)) ** 2 + (b * np.sin(d)) ** 2
        rad = np.clip(q - sp * sp, 0.0, None)
        out += rho * 2.0 * a * b * np.sqrt(rad) / q
    return out * (N / 2.0)


def disk_sinogram(radius_px: float, n_angles: int, n_det: int) -> np.ndarray:
    """Line integrals of a centred unit-intensity disk of radius R (pixel
    units): 2*sqrt(R^2 - u^2), independent of the angle."""
    u = np.arange(n_det, dtype=np.float64) - (n_det - 1) / 2.0
    row = 2.0 * np.sqrt(np.clip(radius_px * radius_px - u * u, 0.0, None))
    return np.repeat(row[None, :], n_angles, axis=0)


def noisy_sinogram(y_clean: np.ndarray, N: int, seed: int, I0: float = 1e5,
                   sigma: float = 0.01) -> np.ndarray:
    """Poisson photon noise at I0 plus Gaussian noise of std sigma in physical
    post-log units.  y_clean is in pixel units; kappa = 2/N converts."""
    rng = np.random.default_rng(seed)
    kappa = 2.0 / N
    counts = rng.poisson(I0 * np.exp(-kappa * y_clean))
    post_log = -np.log(np.maximum(counts, 1) / I0)
    post_log = post_log + sigma * rng.standard_normal(y_clean.shape)
    return post_log / kappa


def uniform_angles(n_angles: int) -> np.ndarray:
    """theta_a = 180 a / n_angles degrees, a = 0..n_angles-1."""
    return 180.0 * np.arange(n_angles, dtype=np.float64) / n_angles


def sketch_indices(n_angles: int, m: int, offset: int) -> np.ndarray:
    """Interleaved angle subset S_k = {offset + j*stride}, stride = n_angles/m
    (Sec. 4.2.1: the operator is split into N interleaved minibatches)."""
    if m <= 0 or n_angles % m != 0:
        raise ValueError("sketch size must divide the angle count")
    stride = n_angles // m
    if not 0 <= offset < stride:
        raise ValueError("offset must lie in [0, stride)")
    return (offset + stride * np.arange(m)).astype(np.int32)


def random_sketch_offset(rng: np.random.Generator, n_angles: int, m: int) -> int:
    return int(rng.integers(0, n_angles // m))


def rotation_angles(rng: np.random.Generator, B: int, G: int) -> np.ndarray:
    """G rotation angles per sample, U[0, 360) degrees, float64 [B, G]."""
    return rng.uniform(0.0, 360.0, size=(B, G))


def step_rng(step: int) -> np.random.Generator:
    """Per-iteration randomness (sketch offset, rotations)."""
    return np.random.default_rng(1000 + int(step))


# --------------------------------------------------------------------------
# weights of the residual CNN that stands in for the paper's pre-trained
# network in BN-only test-time training (Sec. 3.3); the paper's U-Net and
# its trained weights are not available, so both sides build the same
# seeded network from these arrays
# --------------------------------------------------------------------------

@dataclass
class CnnWeights:
    conv: list        # float64 [C_out, C_in, 3, 3] per layer: 1 -> C, C -> C ..., C -> 1
    bn: np.ndarray    # float64 [2 C (L-1)]: per BN layer l, scale[C] then shift[C]
    channels: int
    layers: int


def cnn_weights(channels: int = 16, layers: int = 4, seed: int = 0) -> CnnWeights:
    """He-normal 3x3 kernels (std sqrt(2 / (9 C_in))), the last layer scaled
    by 0.1 so that the residual branch starts small; BN scales drawn around 1
    and shifts around 0, as after pre-training."""
    if layers < 2 or channels < 1:
        raise ValueError("need layers >= 2 and channels >= 1")
    rng = np.random.default_rng(seed)
    chans = [1] + [channels] * (layers - 1) + [1]
    conv = []
    for l in range(layers):
        cin, cout = chans[l], chans[l + 1]
        w = rng.standard_normal((cout, cin, 3, 3)) * math.sqrt(2.0 / (9 * cin))
        conv.append(w * (0.1 if l == layers - 1 else 1.0))
    bn = []
    for _ in range(layers - 1):
        bn.append(1.0 + 0.1 * rng.standard_normal(channels))
        bn.append(0.1 * rng.standard_normal(channels))
    return CnnWeights(conv=conv, bn=np.concatenate(bn), channels=channels, layers=layers)


# --------------------------------------------------------------------------
# multi-coil MRI stand-ins (Sec. 4.1.2: 15-coil knee k-space at 128 x 128,
# 4x undersampling; the fastMRI data and ESPIRiT maps are not available)
# --------------------------------------------------------------------------

def complex_phantom(seed: int, N: int) -> np.ndarray:
    """Planar complex image [2, N, N]: an ellipse phantom's magnitude times a
    smooth random phase (low-order polynomial, |phase| < pi/2)."""
    rng = np.random.default_rng(seed + 5000)
    mag = rasterize(random_ellipses(seed), N)
    y, x = np.meshgrid(np.linspace(-1, 1, N), np.linspace(-1, 1, N), indexing="ij")
    a = rng.uniform(-0.5, 0.5, size=4)
    ph = a[0] * x + a[1] * y + a[2] * x * y + a[3] * (x * x - y * y)
    return np.stack([mag * np.cos(ph), mag * np.sin(ph)])


def coil_maps(Nc: int, N: int, seed: int = 0) -> np.ndarray:
    """Planar sensitivity maps [Nc, 2, N, N]: coil c sits on a circle of
    radius 1.5 (field of view [-1, 1]^2) at angle 2 pi c / Nc; magnitude
    exp(-|r - r_c|^2 / (2 w^2)) with w = 0.9, phase = the polar angle seen from
    the coil plus a seeded constant."""
    rng = np.random.default_rng(seed + 6000)
    y, x = np.meshgrid(np.linspace(-1, 1, N), np.linspace(-1, 1, N), indexing="ij")
    maps = np.zeros((Nc, 2, N, N))
    for c in range(Nc):
        t = 2 * np.pi * c / Nc
        cx, cy = 1.5 * np.cos(t), 1.5 * np.sin(t)
        mag = np.exp(-((x - cx) ** 2 + (y - cy) ** 2) / (2 * 0.9 ** 2))
        ph = np.arctan2(y - cy, x - cx) + rng.uniform(0, 2 * np.pi)
        maps[c, 0], maps[c, 1] = mag * np.cos(ph), mag * np.sin(ph)
    return maps


def undersampling_mask(N: int, accel: int = 4, center: float = 0.08, seed: int = 0) -> np.ndarray:
    """[N, N] 0/1 mask of whole k-space lines along the first axis (frequency
    0 at index 0, no shift): the ceil(center N) lowest |frequencies| plus
    random others, N / accel lines in all."""
    rng = np.random.default_rng(seed + 7000)
    freq = np.fft.fftfreq(N) * N
    order = np.argsort(np.abs(freq), kind="stable")
    n_c = int(np.ceil(center * N))
    n_all = max(n_c, N // accel)
    lines = list(order[:n_c])
    rest = order[n_c:]
    lines += list(rng.choice(rest, size=n_all - n_c, replace=False))
    m = np.zeros((N, N))
    m[np.array(lines, dtype=np.int64)] = 1.0
    return m


def rademacher(rng: np.random.Generator, shape) -> np.ndarray:
    """i.i.d. +-1 with probability 1/2."""
    return rng.integers(0, 2, size=shape) * 2.0 - 1.0
