"""The measurement noise model of the seeded inputs (Poisson photon counts
at I0 plus Gaussian noise of std sigma after the log, in physical units
kappa = 2/N per pixel), checked against its statistics: by the delta method
the post-log value has mean kappa y + 1/(2 lambda) and variance 1/lambda +
sigma^2, lambda = I0 exp(-kappa y)."""
import numpy as np
import pytest

from paper_2411_05771_gb300 import inputs as I


@pytest.mark.parametrize("kappa_y,sigma", [(1.0, 0.01), (0.0, 0.01), (2.0, 0.0)])
def test_noise_mean_and_variance(kappa_y, sigma):
    N, I0, n = 256, 1e5, 400_000
    kappa = 2.0 / N
    y = np.full(n, kappa_y / kappa)
    z = I.noisy_sinogram(y, N, seed=17, I0=I0, sigma=sigma)
    lam = I0 * np.exp(-kappa_y)
    var = (1.0 / lam + sigma ** 2) / kappa ** 2
    mean = y[0] + 1.0 / (2.0 * lam * kappa)
    assert abs(z.mean() - mean) < 5.0 * np.sqrt(var / n)
    assert abs(z.var() / var - 1.0) < 5.0 * np.sqrt(2.0 / n)


def test_noise_is_seeded():
    y = np.linspace(0.0, 300.0, 1000)
    a = I.noisy_sinogram(y, 256, seed=3)
    assert np.array_equal(a, I.noisy_sinogram(y, 256, seed=3))
    assert not np.array_equal(a, I.noisy_sinogram(y, 256, seed=4))
