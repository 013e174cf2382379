"""Seeded synthetic workloads for the D-NGD step.

This module only draws inputs: collocation points, target values of the
manufactured solutions, initial parameters and landmark indices.  It holds
none of the method's arithmetic (no jets, Jacobians, Gramians or solves) and
is the one module that both the CUDA path's callers and the CPU oracle's
callers read their inputs from.

A workload is a plain dict:

    widths   layer widths [d_in, w_1, ..., w_L, 1]
    classes  list of {count, c_val, c_grad[d], c_lap, lap_mask[d]}: the
             residual class sizes and the linear operator of each class,
             Op u = c_val u + sum_k c_grad[k] d_k u + c_lap sum_{k in mask} d_kk u
    X        [m, d] float64 collocation points, classes in order
    target   [m] float64 right-hand sides (f inside, g on boundary/initial)
    theta    [n] float64 initial parameters (Glorot-uniform, zero biases)
    lam      damping

Sampling readings (the paper says "uniform" without more detail): points are
i.i.d. uniform; square boundaries use equal counts per edge; cube boundaries
pick a face uniformly among the 2d faces and the other coordinates uniformly.
Seeds: theta uses ``seed``, the points ``seed + 1``.
"""
import math

import numpy as np


def n_params(widths):
    return int(sum(widths[l] * widths[l - 1] + widths[l] for l in range(1, len(widths))))


def glorot_theta(widths, seed):
    """Glorot-uniform weights U(+-sqrt(6/(fan_in+fan_out))), zero biases,
    drawn layer by layer (W row-major) from numpy default_rng(seed)."""
    rng = np.random.default_rng(seed)
    parts = []
    for l in range(1, len(widths)):
        fi, fo = widths[l - 1], widths[l]
        a = math.sqrt(6.0 / (fi + fo))
        parts.append(rng.uniform(-a, a, size=fo * fi))
        parts.append(np.zeros(fo))
    return np.concatenate(parts)


def _poisson_classes(d, n_int, n_bnd):
    return [
        dict(count=int(n_int), c_val=0.0, c_grad=[0.0] * d, c_lap=-1.0, lap_mask=[1] * d),
        dict(count=int(n_bnd), c_val=1.0, c_grad=[0.0] * d, c_lap=0.0, lap_mask=[0] * d),
    ]


def square_boundary(n, rng):
    """n points on the boundary of [0,1]^2, n/4 per edge (remainder spread
    over the first edges)."""
    counts = [n // 4 + (1 if e < n % 4 else 0) for e in range(4)]
    pts = []
    for e, c in enumerate(counts):
        s = rng.uniform(0.0, 1.0, size=c)
        if e == 0:
            pts.append(np.stack([s, np.zeros(c)], 1))
        elif e == 1:
            pts.append(np.stack([s, np.ones(c)], 1))
        elif e == 2:
            pts.append(np.stack([np.zeros(c), s], 1))
        else:
            pts.append(np.stack([np.ones(c), s], 1))
    return np.concatenate(pts, 0)


def cube_boundary(n, d, rng):
    """n points on the boundary of [0,1]^d: a face is chosen uniformly among
    the 2d faces, the other coordinates are uniform."""
    X = rng.uniform(0.0, 1.0, size=(n, d))
    face = rng.integers(0, 2 * d, size=n)
    X[np.arange(n), face // 2] = (face % 2).astype(np.float64)
    return X


def poisson_sine(d, widths, n_int, n_bnd, k=1, seed=0, lam=1e-8, product=None):
    """-Laplace(u) = f on [0,1]^d with a sine manufactured solution.

    product=True  : u = prod_i sin(k pi x_i)  (vanishes on the boundary, g = 0)
    product=False : u = sum_i sin(k pi x_i)   (g = u on the boundary)
    Default: product form in 2-D, sum form otherwise."""
    if product is None:
        product = (d == 2)
    rng = np.random.default_rng(seed + 1)
    Xi = rng.uniform(0.0, 1.0, size=(n_int, d))
    Xb = square_boundary(n_bnd, rng) if d == 2 else cube_boundary(n_bnd, d, rng)
    kp = k * math.pi
    if product:
        f = d * kp * kp * np.prod(np.sin(kp * Xi), axis=1)
        g = np.zeros(n_bnd)          # the product form vanishes on the boundary
    else:
        f = kp * kp * np.sum(np.sin(kp * Xi), axis=1)
        g = np.sum(np.sin(kp * Xb), axis=1)
    return dict(
        name=f"poisson{d}d", widths=list(widths), classes=_poisson_classes(d, n_int, n_bnd),
        X=np.concatenate([Xi, Xb], 0), target=np.concatenate([f, g]),
        theta=glorot_theta(widths, seed), lam=float(lam), k=int(k), product=bool(product))


def heat_1d(widths, n_int, n_bnd, n_init, kappa=0.1, seed=0, lam=1e-5):
    """u_t = kappa u_xx on (t, x) in [0,1]^2, u(0,x) = sin(pi x), u(t,0) =
    u(t,1) = 0.  Inputs are ordered (t, x); three residual classes."""
    rng = np.random.default_rng(seed + 1)
    Xi = rng.uniform(0.0, 1.0, size=(n_int, 2))
    tb = rng.uniform(0.0, 1.0, size=n_bnd)
    xb = np.concatenate([np.zeros(n_bnd // 2), np.ones(n_bnd - n_bnd // 2)])
    Xb = np.stack([tb, xb], 1)
    x0 = rng.uniform(0.0, 1.0, size=n_init)
    X0 = np.stack([np.zeros(n_init), x0], 1)
    classes = [
        dict(count=int(n_int), c_val=0.0, c_grad=[1.0, 0.0], c_lap=-float(kappa), lap_mask=[0, 1]),
        dict(count=int(n_bnd), c_val=1.0, c_grad=[0.0, 0.0], c_lap=0.0, lap_mask=[0, 0]),
        dict(count=int(n_init), c_val=1.0, c_grad=[0.0, 0.0], c_lap=0.0, lap_mask=[0, 0]),
    ]
    target = np.concatenate([np.zeros(n_int), np.zeros(n_bnd), np.sin(math.pi * x0)])
    return dict(name="heat1d", widths=list(widths), classes=classes,
                X=np.concatenate([Xi, Xb, X0], 0), target=target,
                theta=glorot_theta(widths, seed), lam=float(lam), kappa=float(kappa))


# --------------------------------------------------------------------------
# The five benchmark workloads
# --------------------------------------------------------------------------

def poisson2d_fp64(seed=0):
    """2-D Poisson, u = sin(pi x) sin(pi y), MLP 2-32-32-1 (n = 1,185),
    400 interior + 100 boundary points, lambda = 1e-8."""
    return poisson_sine(2, [2, 32, 32, 1], 400, 100, k=1, seed=seed, lam=1e-8)


def poisson5d_dense(seed=0, lam=1e-8):
    """5-D Poisson, u = sum sin(pi x_i), MLP 5-256-256-256-1 (n = 133,377),
    3,000 interior + 1,000 boundary points (m = 4,000)."""
    return poisson_sine(5, [5, 256, 256, 256, 1], 3000, 1000, k=1, seed=seed, lam=lam)


def heat_pcg(seed=0, width=2048, depth=4, lam=1e-5):
    """1+1-D heat, kappa = 0.1, MLP 2-2048x4-1 (n = 12,597,249), 6,144
    interior + 1,024 boundary + 1,024 initial points (m = 8,192)."""
    return heat_1d([2] + [width] * depth + [1], 6144, 1024, 1024, kappa=0.1, seed=seed, lam=lam)


def landmarks(m, ell, seed):
    """Landmark residual indices: the first ell entries of a seeded
    permutation of 0..m-1, sorted."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.permutation(m)[:ell]).astype(np.int64)


def poisson2d_batch(n_inst=64, seed=0, lam=1e-8):
    """64 independent 2-D Poisson instances: k ~ U{1..8}, width ~ U{32,64,128}
    (two hidden layers), m ~ U[256, 2048] with N_boundary = round(0.2 m).
    Instance b uses seed 1000 + b."""
    out = []
    for b in range(n_inst):
        rng = np.random.default_rng(1000 + b + seed)
        k = int(rng.integers(1, 9))
        w = int(rng.choice([32, 64, 128]))
        m = int(rng.integers(256, 2049))
        nb = int(round(0.2 * m))
        out.append(poisson_sine(2, [2, w, w, 1], m - nb, nb, k=k, seed=1000 + b + seed, lam=lam))
    return out


def serving_jobs(n_jobs, rate_per_s=200.0, seed=7, lam=1e-5, m_range=(512, 8192),
                 widths=(64, 128, 256, 512), depths=(2, 3), n_steps=50):
    """Arrival stream of PINN solve jobs: exponential inter-arrival times
    (mean 1/rate), 2-D / 5-D Poisson 50/50, k ~ U{1..8}, m ~ U[m_range],
    width ~ U{widths}, depth ~ U{depths}.  Returns a list of
    (arrival_time_s, workload, n_steps)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    jobs = []
    for j in range(n_jobs):
        t += float(rng.exponential(1.0 / rate_per_s))
        d = 2 if rng.uniform() < 0.5 else 5
        k = int(rng.integers(1, 9))
        m = int(rng.integers(m_range[0], m_range[1] + 1))
        w = int(rng.choice(list(widths)))
        depth = int(rng.choice(list(depths)))
        nb = int(round(0.2 * m))
        wl = poisson_sine(d, [d] + [w] * depth + [1], m - nb, nb, k=k, seed=10000 + j, lam=lam)
        jobs.append((t, wl, int(n_steps)))
    return jobs
