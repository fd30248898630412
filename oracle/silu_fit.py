"""Task-specific SiLU approximation (test infrastructure only).

Range (Eq. 11, Chebyshev's inequality with eps = 5 sigma):
    [max(mu - 5 sigma, x_min), min(mu + 5 sigma, x_max)].
Fit (Eq. 12): weighted least squares over points sampled uniformly in the
range, weight 10 inside [mu - 3 sigma, mu + 3 sigma] and 1 outside.

Readings where the paper is silent: the samples are an evenly spaced grid of
`n_samples` points including both ends; the polynomial is expressed in the
Chebyshev basis of the range mapped to [-1, 1]; the least-squares problem is
solved by Householder QR of the row-weighted design matrix.
"""
import numpy as np

from .kan_plain import silu


def silu_range(mu, sigma, x_min, x_max):
    return max(mu - 5.0 * sigma, x_min), min(mu + 5.0 * sigma, x_max)


def wls_weights(x, mu, sigma):
    return np.where(np.abs(x - mu) <= 3.0 * sigma, 10.0, 1.0)


def fit_silu(lo, hi, mu, sigma, degree, n_samples=10000):
    """Chebyshev coefficients a_0..a_d of the weighted least-squares fit."""
    x = np.linspace(lo, hi, n_samples)
    y = (2.0 * x - (lo + hi)) / (hi - lo)
    V = np.polynomial.chebyshev.chebvander(y, degree)
    sw = np.sqrt(wls_weights(x, mu, sigma))
    Q, Rm = np.linalg.qr(V * sw[:, None])
    return np.linalg.solve(Rm, Q.T @ (silu(x) * sw))


def layer_stats(acts):
    """mu, sigma, min, max of a layer's SiLU inputs over a calibration set."""
    a = np.asarray(acts, dtype=np.float64).ravel()
    return float(a.mean()), float(a.std()), float(a.min()), float(a.max())
