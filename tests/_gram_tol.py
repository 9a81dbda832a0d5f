"""Tolerances of the GPU statistics against the oracle's that come from the reduction's
arithmetic. The Gram of the statistics kernel forms each per-site product from BF16 hi + lo
splits of both factors: each factor keeps a residual below 2^-16 of itself (the rounding
of its lo part, of either sign), so a product carries at most 2^-15 relative error, with
random sign from site to site. A sum over N sites of terms x_s then deviates by about
2^-15 sqrt(sum x_s^2); the bounds below take six times that (the FP64 oracle has none)."""
import numpy as np

EPS = 2.0 ** -15


def sum_tol(sum_of_squares):
    """Bound on |GPU - oracle| for a sum of per-site terms with the given sum of squares."""
    return 6.0 * EPS * np.sqrt(sum_of_squares)


def mean_tol(mean_of_squares, n):
    """The same bound for a mean over n sites, from the mean of the squared terms."""
    return 6.0 * EPS * np.sqrt(np.asarray(mean_of_squares, dtype=float) / n)


def uu_tol(uu, n):
    """Bounds for <u_a u_b> (xx, yy, zz, xy, xz, yz) from the diagonal means <u_a^2>, with
    <u_a^2 u_b^2> taken as 3 <u_a^2> <u_b^2> (its Gaussian value for a = b)."""
    d = np.asarray(uu[:3], dtype=float)
    pairs = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    return np.array([mean_tol(3.0 * d[a] * d[b], n) for a, b in pairs])
