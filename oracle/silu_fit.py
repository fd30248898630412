"""Task-specific SiLU approximation (test infrastructure only).

Range (Eq. 11, Chebyshev's inequality with eps = 5 sigma):
    [max(mu - 5 sigma, x_min), min(mu + 5 sigma, x_max)].
Fit (Eq. 12): weighted least squares over points sampled uniformly in the
range, weight 10 inside [mu - 3 sigma, mu + 3 sigma] and 1 outside.

Readings where the paper is silent: the samples are an evenly spaced grid of
`n_samples` points including both ends; the polynomial is expressed in the
Chebyshev basis of the range mapped to [-1, 1]; the least-squares problem is
solved by Householder QR of the row-weighted design matrix.

The two methods the paper compares against (Table 5), on the same range and
degree: OLS, the same least squares with unit weights; Remez, the minimax
polynomial by the Remez exchange (reference of d + 2 points starting at the
Chebyshev extrema; solve p(x_i) + (-1)^i E = f(x_i); move the reference to
the d + 2 alternating extrema of the error on the sample grid, dropping the
smaller end run while there are more; stop when the reference repeats).
"""
import numpy as np

from .kan_plain import silu


def silu_range(mu, sigma, x_min, x_max):
    return max(mu - 5.0 * sigma, x_min), min(mu + 5.0 * sigma, x_max)


def wls_weights(x, mu, sigma):
    return np.where(np.abs(x - mu) <= 3.0 * sigma, 10.0, 1.0)


def fit_silu(lo, hi, mu, sigma, degree, n_samples=10000, method="wls", f=silu):
    """Chebyshev coefficients a_0..a_d (basis of [lo, hi] mapped to [-1, 1])
    of the weighted least-squares fit (Eq. 12), of OLS or of Remez."""
    x = np.linspace(lo, hi, n_samples)
    y = (2.0 * x - (lo + hi)) / (hi - lo)
    if method == "remez":
        return remez(lambda t: f(0.5 * (hi - lo) * t + 0.5 * (hi + lo)), degree, y)
    V = np.polynomial.chebyshev.chebvander(y, degree)
    w = wls_weights(x, mu, sigma) if method == "wls" else np.ones_like(x)
    sw = np.sqrt(w)
    Q, Rm = np.linalg.qr(V * sw[:, None])
    return np.linalg.solve(Rm, Q.T @ (f(x) * sw))


def _runs(e):
    """(start, end) of the maximal runs of equal sign of e (zeros join the
    run before them)."""
    sg = np.sign(e)
    for i in range(1, len(sg)):
        if sg[i] == 0:
            sg[i] = sg[i - 1]
    out, st = [], 0
    for i in range(1, len(sg) + 1):
        if i == len(sg) or sg[i] != sg[st]:
            out.append((st, i))
            st = i
    return out


def remez(g, degree, grid, max_iter=60):
    """Minimax Chebyshev coefficients of g on [-1, 1] over the points `grid`."""
    n = degree + 2
    ref = -np.cos(np.pi * np.arange(n) / (n - 1))
    c = np.zeros(degree + 1)
    prev = None
    for _ in range(max_iter):
        A = np.zeros((n, n))
        A[:, :degree + 1] = np.polynomial.chebyshev.chebvander(ref, degree)
        A[:, degree + 1] = (-1.0) ** np.arange(n)
        sol = np.linalg.solve(A, g(ref))
        c = sol[:degree + 1]
        e = g(grid) - np.polynomial.chebyshev.chebval(grid, c)
        runs = [(a + int(np.argmax(np.abs(e[a:b]))), float(np.abs(e[a:b]).max())) for a, b in _runs(e)]
        if len(runs) < n:
            break
        while len(runs) > n:
            runs.pop(0 if runs[0][1] < runs[-1][1] else -1)
        idx = [i for i, _ in runs]
        if idx == prev:
            break
        prev = idx
        ref = grid[idx]
    return c


def layer_stats(acts):
    """mu, sigma, min, max of a layer's SiLU inputs over a calibration set."""
    a = np.asarray(acts, dtype=np.float64).ravel()
    return float(a.mean()), float(a.std()), float(a.min()), float(a.max())
