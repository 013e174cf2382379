"""PINN residual map r(theta), its Jacobian J, J v and f_vv (Sec. 2.1-2.2, 3.2).

Residual (Sec. 2.2): the m residuals are grouped by class gamma (interior,
boundary, initial ...) in that order; each class has N_gamma points and

    r_gamma(theta)_i = (Op_gamma u_theta(x_i) - target_i) / sqrt(N_gamma).

Every operator used here is linear in the jets of u:

    Op u = c_val * u + sum_k c_grad[k] * d_k u + c_lap * sum_{k in mask} d_kk u

which covers -Laplace(u) (c_lap = -1, mask = all), Dirichlet data (c_val = 1)
and the heat operator u_t - kappa u_xx (c_grad[t] = 1, c_lap = -kappa,
mask = {x}).  The loss is L = 1/2 ||r||^2 (Eq. pinn_loss).

Two independent derivations live here:
* ``forward_series`` runs one truncated bivariate Taylor series per needed
  coordinate (Taylor-mode AD, Sec. 5) and gives r, J v and f_vv.
* ``residual_and_jacobian`` computes r and the full J by per-point reverse
  mode through the univariate coordinate 2-jets (value, d_k, d_kk/2).
They are cross-checked against each other and against finite differences in
the test-suite.
"""
from dataclasses import dataclass, field

import numpy as np

from . import mlp, series


@dataclass
class ClassOp:
    """One residual class: N points and the linear operator applied to u."""
    count: int
    c_val: float = 0.0
    c_grad: tuple = ()          # length d (empty means all zero)
    c_lap: float = 0.0
    lap_mask: tuple = ()        # length d booleans (empty means none)

    def grad(self, d):
        return np.zeros(d) if len(self.c_grad) == 0 else np.asarray(self.c_grad, dtype=np.float64)

    def mask(self, d):
        return np.zeros(d, dtype=bool) if len(self.lap_mask) == 0 else np.asarray(self.lap_mask, dtype=bool)

    def coords(self, d):
        """Coordinates whose first or second derivative the operator needs."""
        g, msk = self.grad(d), self.mask(d)
        return [k for k in range(d) if g[k] != 0.0 or (msk[k] and self.c_lap != 0.0)]


@dataclass
class Problem:
    widths: list
    classes: list = field(default_factory=list)

    @property
    def d(self):
        return self.widths[0]

    @property
    def m(self):
        return int(sum(c.count for c in self.classes))

    @property
    def n(self):
        return mlp.n_params(self.widths)

    def class_slices(self):
        out, off = [], 0
        for c in self.classes:
            out.append((c, slice(off, off + c.count)))
            off += c.count
        return out


def problem_from_spec(spec):
    """Build a Problem from a workload dict (widths + class list)."""
    cls = []
    for c in spec["classes"]:
        cls.append(ClassOp(int(c["count"]), float(c["c_val"]), tuple(float(g) for g in c["c_grad"]),
                           float(c["c_lap"]), tuple(bool(b) for b in c["lap_mask"])))
    return Problem(list(spec["widths"]), cls)


def poisson_problem(widths, n_interior, n_boundary):
    """-Laplace(u) = f inside, u = g on the boundary (Sec. 2.1)."""
    d = widths[0]
    return Problem(list(widths), [
        ClassOp(n_interior, c_lap=-1.0, lap_mask=tuple([True] * d)),
        ClassOp(n_boundary, c_val=1.0),
    ])


def heat_problem(widths, kappa, n_interior, n_boundary, n_initial):
    """u_t - kappa u_xx = 0 on (t, x) in [0,1]^2; inputs are ordered (t, x).
    Three classes (interior, boundary, initial), each with its own scale."""
    assert widths[0] == 2
    return Problem(list(widths), [
        ClassOp(n_interior, c_grad=(1.0, 0.0), c_lap=-float(kappa), lap_mask=(False, True)),
        ClassOp(n_boundary, c_val=1.0),
        ClassOp(n_initial, c_val=1.0),
    ])


# ---------------------------------------------------------------------------
# Forward Taylor-mode pass (r, J v, f_vv)
# ---------------------------------------------------------------------------

def _network_series(layers, dirs, h):
    """Propagate a series through the MLP.  ``dirs`` gives (V_l, bv_l) per
    layer or None."""
    L = len(layers)
    for l, (W, b) in enumerate(layers):
        V, bv = (None, None) if dirs is None else dirs[l]
        h = series.affine(W, b, V, bv, h)
        if l < L - 1:
            h = series.tanh(h)
    return h[..., 0]          # output width is 1


def forward_series(theta, problem, X, target, v=None):
    """Return (r, Jv, f_vv) by Taylor-mode series along each needed spatial
    coordinate and along the parameter direction v (Sec. 3.2, Sec. 5).
    With v None, Jv and f_vv are zero."""
    X = np.asarray(X, dtype=np.float64)
    target = np.asarray(target, dtype=np.float64)
    widths = problem.widths
    d = problem.d
    layers = mlp.unpack(theta, widths)
    dirs = None if v is None else mlp.unpack(v, widths)
    m = problem.m
    coef = np.zeros((3, m))        # t-degree coefficients of r
    for cls, sl in problem.class_slices():
        x = X[sl]
        npts = x.shape[0]
        acc = np.zeros((3, npts))  # sum over operator terms, per t-degree
        coords = cls.coords(d)
        # value term (any direction; eps-free part)
        if cls.c_val != 0.0 or not coords:
            h = series.constant(x)
            u = _network_series(layers, dirs, h)
            acc += cls.c_val * u[0, :]
        g, msk = cls.grad(d), cls.mask(d)
        for k in coords:
            h = series.constant(x)
            h[1, 0, :, k] = 1.0            # x + eps e_k
            u = _network_series(layers, dirs, h)
            if g[k] != 0.0:
                acc += g[k] * u[1, :]
            if msk[k] and cls.c_lap != 0.0:
                acc += cls.c_lap * 2.0 * u[2, :]
        acc[0] -= target[sl]
        coef[:, sl] = acc / np.sqrt(cls.count)
    r = coef[0]
    jv = coef[1]
    fvv = 2.0 * coef[2]
    return r, jv, fvv


def second_directional(theta, problem, X, target, v):
    """f_vv = d^2/dt^2 r(theta + t v)|_{t=0} (Sec. 3.2)."""
    return forward_series(theta, problem, X, target, v)[2]


def jvp(theta, problem, X, target, v):
    """J v = d/dt r(theta + t v)|_{t=0}."""
    return forward_series(theta, problem, X, target, v)[1]


# ---------------------------------------------------------------------------
# Reverse mode: r and the full Jacobian J (m x n)
# ---------------------------------------------------------------------------

def _class_rows(layers, cls, d, x, target, scale, J_rows):
    """Residuals and Jacobian rows of one class by per-point reverse mode
    through the coordinate 2-jets.  Writes J_rows [npts, n] in place."""
    npts = x.shape[0]
    coords = cls.coords(d)
    K = len(coords)
    g, msk = cls.grad(d), cls.mask(d)
    L = len(layers)
    # forward: value h0 [npts, w]; per-coordinate h1, h2 [npts, K, w]
    h0 = x.copy()
    h1 = np.zeros((npts, K, d))
    for a, k in enumerate(coords):
        h1[:, a, k] = 1.0
    h2 = np.zeros((npts, K, d))
    saved = []
    for l, (W, b) in enumerate(layers):
        z0 = h0 @ W.T + b
        z1 = h1 @ W.T
        z2 = h2 @ W.T
        saved.append((h0, h1, h2, z0, z1, z2))
        if l < L - 1:
            T = np.tanh(z0)
            s = 1.0 - T * T
            h0 = T
            h1 = s[:, None, :] * z1
            h2 = s[:, None, :] * z2 - (T * s)[:, None, :] * z1 * z1
        else:
            h0, h1, h2 = z0, z1, z2
    u0 = h0[:, 0]
    u1 = h1[:, :, 0]
    u2 = h2[:, :, 0]
    cg = np.array([g[k] for k in coords])
    cl = np.array([cls.c_lap * 2.0 if msk[k] else 0.0 for k in coords])
    r = scale * (cls.c_val * u0 + u1 @ cg + u2 @ cl - target)
    # reverse: adjoints of the output series coefficients
    A0 = np.full((npts, 1), scale * cls.c_val)
    A1 = np.broadcast_to(scale * cg[None, :, None], (npts, K, 1)).copy()
    A2 = np.broadcast_to(scale * cl[None, :, None], (npts, K, 1)).copy()
    col = J_rows.shape[1]
    offs = mlp.layer_offsets([d] + [W.shape[0] for W, _ in layers])
    for l in range(L - 1, -1, -1):
        W, b = layers[l]
        hp0, hp1, hp2, z0, z1, z2 = saved[l]
        if l < L - 1:
            # adjoint through tanh: T0 = t, T1 = s z1, T2 = s z2 - t s z1^2
            T = np.tanh(z0)
            s = 1.0 - T * T
            ts = T * s
            dts = s * (s - 2.0 * T * T)          # d(t s)/dz
            Z2 = s[:, None, :] * A2
            Z1 = s[:, None, :] * A1 - 2.0 * ts[:, None, :] * z1 * A2
            Z0 = s * A0 + np.sum(-2.0 * ts[:, None, :] * z1 * A1
                                 + (-2.0 * ts[:, None, :] * z2 - dts[:, None, :] * z1 * z1) * A2, axis=1)
        else:
            Z0, Z1, Z2 = A0, A1, A2
        wo, bo, o, i = offs[l]
        gW = (np.einsum("pa,pb->pab", Z0, hp0)
              + np.einsum("pka,pkb->pab", Z1, hp1)
              + np.einsum("pka,pkb->pab", Z2, hp2))
        J_rows[:, wo:wo + o * i] = gW.reshape(npts, o * i)
        J_rows[:, bo:bo + o] = Z0
        A0 = Z0 @ W
        A1 = Z1 @ W
        A2 = Z2 @ W
    assert col == J_rows.shape[1]
    return r


def residual_and_jacobian(theta, problem, X, target, chunk=256):
    """Return (r [m], J [m, n]) in float64 (Sec. 2.2; J = d r / d theta)."""
    X = np.asarray(X, dtype=np.float64)
    target = np.asarray(target, dtype=np.float64)
    layers = mlp.unpack(theta, problem.widths)
    d = problem.d
    r = np.zeros(problem.m)
    J = np.zeros((problem.m, problem.n))
    for cls, sl in problem.class_slices():
        scale = 1.0 / np.sqrt(cls.count)
        for p0 in range(sl.start, sl.stop, chunk):
            p1 = min(sl.stop, p0 + chunk)
            r[p0:p1] = _class_rows(layers, cls, d, X[p0:p1], target[p0:p1], scale, J[p0:p1])
    return r, J


def residual(theta, problem, X, target):
    """r(theta) only (value pass of the series forward)."""
    return forward_series(theta, problem, X, target, None)[0]


def loss(theta, problem, X, target):
    """L(theta) = 1/2 ||r(theta)||^2 (Sec. 2.2)."""
    r = residual(theta, problem, X, target)
    return 0.5 * float(r @ r)
