"""Pins for the oracle's jets, residuals, Jacobian and f_vv (CPU only).

Each test checks the oracle against something other than itself: values the
paper prints, closed forms, symbolic differentiation, or finite differences.
"""
import os

import numpy as np
import pytest

from oracle import mlp, residual as res, series

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _rng(seed=0):
    return np.random.default_rng(seed)


def _rand_theta(widths, seed=0, scale=0.8):
    return _rng(seed).normal(0.0, scale, size=mlp.n_params(widths))


def _u_values(theta, widths, X):
    """u_theta(X) through the oracle: a value-only class with target 0 and
    count 1 per evaluation (scale 1)."""
    out = []
    for x in np.atleast_2d(X):
        prob = res.Problem(list(widths), [res.ClassOp(1, c_val=1.0)])
        out.append(res.residual(theta, prob, x[None, :], np.zeros(1))[0])
    return np.array(out)


# -- paper-printed parameter counts (Sec. 5, App. A.3) -----------------------

def test_param_counts_match_paper():
    rows = []
    with open(os.path.join(GOLDEN, "paper_param_counts.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            w, n, kind = [p.strip() for p in line.split(";")]
            rows.append(([int(a) for a in w.split(",")], int(n), kind))
    assert len(rows) == 6
    for widths, n, kind in rows:
        got = mlp.n_params(widths)
        if kind == "exact":
            assert got == n, (widths, got, n)
        else:
            assert abs(got - n) / n < 0.02, (widths, got, n)


def test_pack_unpack_roundtrip():
    widths = [3, 4, 5, 1]
    th = _rand_theta(widths)
    assert np.array_equal(mlp.pack(mlp.unpack(th, widths)), th)
    # layout: W_1 row-major then b_1
    W1, b1 = mlp.unpack(th, widths)[0]
    assert W1[1, 2] == th[1 * 3 + 2] and b1[0] == th[12]


# -- tanh derivatives (used by the series arithmetic) ------------------------

def test_tanh_derivatives_vs_sympy():
    sp = pytest.importorskip("sympy")
    z = sp.Symbol("z")
    exprs = [sp.tanh(z)]
    for _ in range(4):
        exprs.append(sp.diff(exprs[-1], z))
    for z0 in [-2.3, -0.4, 0.0, 0.7, 1.9]:
        got = series.tanh_derivatives(np.float64(z0))
        for k in range(5):
            ref = float(exprs[k].subs(z, z0).evalf(30))
            assert abs(got[k] - ref) <= 1e-14 * (1 + abs(ref)), (k, z0)


def test_series_tanh_composition_vs_direct_evaluation():
    # tanh of a bivariate polynomial: compare coefficients with a 2-D
    # polynomial fit of tanh(p(eps, t)) on a tiny grid (exact interpolation
    # of the degree-(2,2) truncation is not available, so use derivatives by
    # central differences of the composed function).
    c = _rng(3).normal(size=(3, 3)) * 0.3
    def f(e, t):
        p = sum(c[i, j] * e ** i * t ** j for i in range(3) for j in range(3))
        return np.tanh(p)
    s = series.tanh(c.reshape(3, 3))
    h = 1e-3
    # d/de, d/dt, d2/de2, d2/dt2, d2/dedt at 0 vs coefficients
    fe = (f(h, 0) - f(-h, 0)) / (2 * h)
    ft = (f(0, h) - f(0, -h)) / (2 * h)
    fee = (f(h, 0) - 2 * f(0, 0) + f(-h, 0)) / h ** 2
    ftt = (f(0, h) - 2 * f(0, 0) + f(0, -h)) / h ** 2
    fet = (f(h, h) - f(h, -h) - f(-h, h) + f(-h, -h)) / (4 * h * h)
    assert abs(s[0, 0] - np.tanh(c[0, 0])) < 1e-15
    assert abs(s[1, 0] - fe) < 1e-6 and abs(s[0, 1] - ft) < 1e-6
    assert abs(2 * s[2, 0] - fee) < 1e-6 and abs(2 * s[0, 2] - ftt) < 1e-6
    assert abs(s[1, 1] - fet) < 1e-6


# -- closed forms ------------------------------------------------------------

def test_laplacian_one_hidden_layer_closed_form():
    # Laplace[c . tanh(W x + b)] = sum_k c_k (-2 t_k (1 - t_k^2)) ||W_k,:||^2
    d, w = 4, 7
    widths = [d, w, 1]
    th = _rand_theta(widths, seed=5)
    (W, b), (C, c0) = mlp.unpack(th, widths)
    X = _rng(6).uniform(size=(9, d))
    prob = res.Problem(widths, [res.ClassOp(9, c_lap=1.0, lap_mask=tuple([True] * d))])
    lap = res.residual(th, prob, X, np.zeros(9)) * 3.0          # undo 1/sqrt(9)
    t = np.tanh(X @ W.T + b)
    ref = ((-2.0 * t * (1 - t * t)) * np.sum(W * W, axis=1)[None, :]) @ C[0]
    assert np.max(np.abs(lap - ref)) <= 1e-13 * (1 + np.max(np.abs(ref)))


def test_linear_network_has_zero_laplacian_and_exact_gradient():
    # With zero hidden layers u = c . x + c0: grad = c, Laplacian = 0.
    d = 3
    widths = [d, 1]
    th = _rand_theta(widths, seed=9)
    X = _rng(1).uniform(size=(4, d))
    prob = res.Problem(widths, [res.ClassOp(4, c_grad=(1.0, 0.0, 0.0), c_lap=1.0, lap_mask=(True,) * 3)])
    r = res.residual(th, prob, X, np.zeros(4)) * 2.0
    assert np.allclose(r, th[0], atol=1e-15)


def test_jets_vs_fourth_order_finite_differences():
    d = 3
    widths = [d, 6, 5, 1]
    th = _rand_theta(widths, seed=2)
    X = _rng(4).uniform(size=(5, d))
    h = 2e-3
    for x in X:
        grad_fd, lap_fd = np.zeros(d), 0.0
        for k in range(d):
            e = np.zeros(d); e[k] = h
            u = _u_values(th, widths, np.stack([x - 2 * e, x - e, x, x + e, x + 2 * e]))
            grad_fd[k] = (u[0] - 8 * u[1] + 8 * u[3] - u[4]) / (12 * h)
            lap_fd += (-u[0] + 16 * u[1] - 30 * u[2] + 16 * u[3] - u[4]) / (12 * h * h)
        for k in range(d):
            cg = [0.0] * d; cg[k] = 1.0
            prob = res.Problem(widths, [res.ClassOp(1, c_grad=tuple(cg))])
            assert abs(res.residual(th, prob, x[None], np.zeros(1))[0] - grad_fd[k]) < 1e-9
        prob = res.Problem(widths, [res.ClassOp(1, c_lap=1.0, lap_mask=(True,) * d)])
        assert abs(res.residual(th, prob, x[None], np.zeros(1))[0] - lap_fd) < 1e-7


def _sympy_net(widths):
    sp = pytest.importorskip("sympy")
    d = widths[0]
    xs = sp.symbols(f"x0:{d}")
    n = mlp.n_params(widths)
    ps = sp.symbols(f"p0:{n}")
    h = list(xs)
    off = 0
    L = len(widths) - 1
    for l in range(1, len(widths)):
        o, i = widths[l], widths[l - 1]
        W = [[ps[off + a * i + b] for b in range(i)] for a in range(o)]
        bb = [ps[off + o * i + a] for a in range(o)]
        off += o * i + o
        z = [sum(W[a][b] * h[b] for b in range(i)) + bb[a] for a in range(o)]
        h = [sp.tanh(v) for v in z] if l < L else z
    return sp, xs, ps, h[0]


def test_residual_jacobian_fvv_vs_sympy():
    """Exact symbolic pins on a tiny net for the heat operator (u_t - k u_xx),
    the Poisson operator and a Dirichlet class: r, full J rows and f_vv."""
    widths = [2, 3, 2, 1]
    sp, xs, ps, u = _sympy_net(widths)
    th = _rand_theta(widths, seed=11)
    v = _rng(12).normal(size=th.size)
    kappa = 0.3
    tsym = sp.Symbol("t")
    ops = {
        "heat": sp.diff(u, xs[0]) - kappa * sp.diff(u, xs[1], 2),
        "poisson": -(sp.diff(u, xs[0], 2) + sp.diff(u, xs[1], 2)),
        "dirichlet": u,
    }
    classes = {
        "heat": res.ClassOp(2, c_grad=(1.0, 0.0), c_lap=-kappa, lap_mask=(False, True)),
        "poisson": res.ClassOp(2, c_lap=-1.0, lap_mask=(True, True)),
        "dirichlet": res.ClassOp(2, c_val=1.0),
    }
    X = _rng(13).uniform(size=(2, 2))
    tgt = np.array([0.25, -0.5])
    for name, expr in ops.items():
        prob = res.Problem(widths, [classes[name]])
        r, J = res.residual_and_jacobian(th, prob, X, tgt)
        r2, jv, fvv = res.forward_series(th, prob, X, tgt, v)
        sc = 1.0 / np.sqrt(2.0)
        for p in range(2):
            e_r = sc * (expr.subs({xs[0]: X[p, 0], xs[1]: X[p, 1]}) - tgt[p])
            f_r = sp.lambdify(ps, e_r, "mpmath")
            rr = float(f_r(*th))
            assert abs(r[p] - rr) < 1e-13 * (1 + abs(rr)), name
            assert abs(r2[p] - rr) < 1e-13 * (1 + abs(rr)), name
            for q in range(0, th.size, 3):
                jr = float(sp.lambdify(ps, sp.diff(e_r, ps[q]), "mpmath")(*th))
                assert abs(J[p, q] - jr) < 1e-12 * (1 + abs(jr)), (name, q)
            # f_vv: second derivative along v of the residual (only t symbolic)
            e_t = e_r.subs({ps[q]: float(th[q]) + tsym * float(v[q]) for q in range(th.size)},
                           simultaneous=True)
            f2 = float(sp.diff(e_t, tsym, 2).subs(tsym, 0).evalf(30))
            assert abs(fvv[p] - f2) < 1e-11 * (1 + abs(f2)), name


# -- reverse-mode J vs forward series and finite differences -----------------

def _poisson(widths, n_int, n_bnd, seed):
    d = widths[0]
    X = np.concatenate([_rng(seed).uniform(size=(n_int, d)),
                        _rng(seed + 1).uniform(size=(n_bnd, d))])
    tgt = _rng(seed + 2).normal(size=n_int + n_bnd)
    return res.poisson_problem(widths, n_int, n_bnd), X, tgt


def test_reverse_jacobian_vs_forward_series_columns():
    widths = [3, 8, 6, 1]
    prob, X, tgt = _poisson(widths, 7, 3, seed=20)
    th = _rand_theta(widths, seed=21)
    r, J = res.residual_and_jacobian(th, prob, X, tgt)
    for q in _rng(22).choice(th.size, size=12, replace=False):
        e = np.zeros(th.size); e[q] = 1.0
        assert np.allclose(res.jvp(th, prob, X, tgt, e), J[:, q], rtol=1e-12, atol=1e-13)
    v = _rng(23).normal(size=th.size)
    jv = res.jvp(th, prob, X, tgt, v)
    assert np.allclose(jv, J @ v, rtol=1e-11, atol=1e-12)
    assert np.allclose(res.residual(th, prob, X, tgt), r, rtol=1e-13, atol=1e-14)


def test_jacobian_vs_central_differences_richardson():
    widths = [2, 5, 4, 1]
    prob = res.heat_problem(widths, 0.1, 4, 2, 2)
    X = _rng(30).uniform(size=(8, 2))
    X[4:6, 1] = [0.0, 1.0]
    X[6:, 0] = 0.0
    tgt = _rng(31).normal(size=8)
    th = _rand_theta(widths, seed=32)
    _, J = res.residual_and_jacobian(th, prob, X, tgt)

    def D(h, q):
        e = np.zeros(th.size); e[q] = h
        return (res.residual(th + e, prob, X, tgt) - res.residual(th - e, prob, X, tgt)) / (2 * h)
    for q in range(th.size):
        h = 1e-3 * max(1.0, abs(th[q]))
        fd = (4 * D(h / 2, q) - D(h, q)) / 3.0
        assert np.allclose(J[:, q], fd, rtol=1e-8, atol=1e-9), q


def test_fvv_vs_central_differences_and_homogeneity():
    widths = [3, 6, 5, 1]
    prob, X, tgt = _poisson(widths, 5, 3, seed=40)
    th = _rand_theta(widths, seed=41)
    v = _rng(42).normal(size=th.size) * 0.3
    fvv = res.second_directional(th, prob, X, tgt, v)

    def S(h):
        return (res.residual(th + h * v, prob, X, tgt) - 2 * res.residual(th, prob, X, tgt)
                + res.residual(th - h * v, prob, X, tgt)) / (h * h)
    fd = (4 * S(5e-4) - S(1e-3)) / 3.0
    assert np.allclose(fvv, fd, rtol=1e-6, atol=1e-7)
    # derivative of the JVP along v: (J(th+hv) v - J(th-hv) v) / 2h
    jp = res.jvp(th + 1e-4 * v, prob, X, tgt, v)
    jm = res.jvp(th - 1e-4 * v, prob, X, tgt, v)
    assert np.allclose(fvv, (jp - jm) / 2e-4, rtol=1e-6, atol=1e-7)
    # homogeneity f_vv(c v) = c^2 f_vv(v)
    assert np.allclose(res.second_directional(th, prob, X, tgt, -2.5 * v), 6.25 * fvv, rtol=1e-12, atol=1e-13)


def test_fvv_zero_for_output_layer_direction():
    # r is affine in the output layer's weights and bias, so its second
    # directional derivative along any output-layer direction vanishes.
    widths = [2, 7, 6, 1]
    prob, X, tgt = _poisson(widths, 6, 4, seed=50)
    th = _rand_theta(widths, seed=51)
    v = np.zeros(th.size)
    nout = widths[-2] + 1
    v[-nout:] = _rng(52).normal(size=nout)
    assert np.max(np.abs(res.second_directional(th, prob, X, tgt, v))) < 1e-13
