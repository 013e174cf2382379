"""Grid line search and parameter update of the D-NGD workflow.

Alg. "D-NGD Workflow" picks eta = argmin_{eta in (0,1]} L(theta + eta dtheta)
and sets theta <- theta + eta dtheta; the hyper-parameter tables (App. A.3)
call it a "31-pt line search".  Reading adopted: the grid is
eta_j = 2^{-j}, j = 0..30, and ties go to the larger eta (the first grid
point in that order).
"""
import numpy as np

from . import residual as res


def grid(k=31):
    return np.array([2.0 ** (-j) for j in range(k)])


def line_search(theta, problem, X, target, delta, etas=None):
    """Return (eta*, losses at every grid point)."""
    etas = grid() if etas is None else np.asarray(etas, dtype=np.float64)
    losses = np.array([res.loss(theta + e * delta, problem, X, target) for e in etas])
    j = int(np.argmin(losses))          # first minimum = largest eta on ties
    return float(etas[j]), losses
