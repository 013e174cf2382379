"""Pins for the oracle's relative L2 error against the manufactured solution.

The midpoint rule on N points integrates sin^2(pi x) over [0,1] exactly
(sum_i sin^2(pi (i + 1/2) / N) = N / 2 for N >= 2) and
sum_i sin(pi (i + 1/2) / N) = 1 / sin(pi / (2N)).  For a network whose output
is the constant c (all weights zero, output bias c) the grid error against
u = sin(pi x) sin(pi y) is therefore, in closed form,
    e = 2 sqrt(c^2 - 2 c mu + 1/4),  mu = (1 / (N sin(pi / (2N))))^2.
"""
import math

import numpy as np

from oracle import evaluate, mlp, residual as res


def test_midpoint_grid_layout():
    g = evaluate.midpoint_grid(2, 3)
    assert g.shape == (9, 2)
    assert np.allclose(g[:3, 1], [1 / 6, 1 / 2, 5 / 6]) and np.allclose(g[:3, 0], 1 / 6)
    assert np.allclose(np.sort(np.unique(g[:, 0])), [1 / 6, 1 / 2, 5 / 6])


def test_constant_network_error_closed_form():
    widths = [2, 5, 4, 1]
    theta = np.zeros(mlp.n_params(widths))
    for N in (4, 17, 64):
        X = evaluate.midpoint_grid(2, N)
        u = evaluate.sine_product(X)
        for c in (0.0, 0.3, -1.2):
            theta[-1] = c                       # output bias
            mu = (1.0 / (N * math.sin(math.pi / (2 * N)))) ** 2
            want = 2.0 * math.sqrt(c * c - 2.0 * c * mu + 0.25)
            assert abs(evaluate.rel_l2_error(theta, widths, X, u) - want) <= 1e-12 * max(1.0, want)


def test_network_values_match_residual_of_value_operator():
    """u_theta(x) equals the residual of the class Op u = u with zero target
    and one point (scale 1), which the residual module computes."""
    widths = [2, 6, 3, 1]
    th = np.random.default_rng(4).normal(0, 0.8, size=mlp.n_params(widths))
    X = np.random.default_rng(5).uniform(size=(7, 2))
    prob = res.Problem(widths, [res.ClassOp(1, c_val=1.0)])
    want = np.array([res.residual(th, prob, X[i:i + 1], np.zeros(1))[0] for i in range(7)])
    assert np.allclose(evaluate.network_values(th, widths, X), want, rtol=1e-14, atol=1e-15)
    # an exact representation has zero error
    assert evaluate.rel_l2_error(th, widths, X, want) <= 1e-15
