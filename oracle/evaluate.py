"""Accuracy of a trained network against the manufactured solution.

The paper reports the relative L2 error of u_theta against the exact solution
on held-out points (Sec. 5, the error columns of its result tables).  This
module evaluates it on a midpoint grid of [0,1]^d:

    e(theta) = sqrt(sum_i (u_theta(x_i) - u(x_i))^2) / sqrt(sum_i u(x_i)^2)

(the grid weights are equal, so the quadrature weight cancels).  Test
infrastructure only; independent of the CUDA path.
"""
import math

import numpy as np

from . import mlp, residual, series


def midpoint_grid(d, N):
    """The N^d midpoints ((i + 1/2) / N, ...) of [0,1]^d, row-major in the
    coordinates (the last coordinate varies fastest)."""
    t = (np.arange(N) + 0.5) / N
    mesh = np.meshgrid(*([t] * d), indexing="ij")
    return np.stack([g.reshape(-1) for g in mesh], axis=1)


def network_values(theta, widths, X):
    """u_theta(x) for every row of X: the value part of the Taylor-mode pass."""
    layers = mlp.unpack(theta, widths)
    h = series.constant(np.asarray(X, dtype=np.float64))
    return residual._network_series(layers, None, h)[0, 0, :]


def sine_product(X, k=1):
    """u(x) = prod_i sin(k pi x_i), the 2-D benchmark's solution."""
    return np.prod(np.sin(k * math.pi * np.asarray(X)), axis=1)


def sine_sum(X, k=1):
    """u(x) = sum_i sin(k pi x_i), the 5-D benchmark's solution."""
    return np.sum(np.sin(k * math.pi * np.asarray(X)), axis=1)


def rel_l2_error(theta, widths, X, u_exact):
    """Relative L2 error of u_theta against u_exact (values at the rows of X)."""
    u = network_values(theta, widths, X)
    return float(np.linalg.norm(u - u_exact) / np.linalg.norm(u_exact))
