"""Truncated bivariate Taylor series: the Taylor-mode arithmetic of the oracle.

The paper computes the spatial derivatives of u_theta with Taylor-mode
automatic differentiation (Sec. 5) and the geodesic-acceleration term with the
second directional derivative f_vv = d^2/dt^2 r(theta + t v)|_{t=0}
(Sec. 3.2).  The oracle carries every scalar of the network as a polynomial

    q(eps, t) = sum_{i<=2, j<=2} c[i, j] eps^i t^j

where ``eps`` moves the input point along one coordinate direction e_k
(x -> x + eps e_k) and ``t`` moves the parameters along a direction v
(theta -> theta + t v).  Hence

    q, d_k q, d_kk q = c[0,0], c[1,0], 2 c[2,0]
    d/dt (.)        = c[.,1]          (a Jacobian-vector product)
    d^2/dt^2 (.)    = 2 c[.,2]        (the f_vv of Sec. 3.2)

Series are NumPy arrays of shape (3, 3) + batch_shape.
"""
import math

import numpy as np

DEG_EPS = 2
DEG_T = 2


def constant(value):
    """Series whose only non-zero coefficient is the constant term."""
    value = np.asarray(value, dtype=np.float64)
    s = np.zeros((DEG_EPS + 1, DEG_T + 1) + value.shape)
    s[0, 0] = value
    return s


def mul(x, y):
    """Truncated product: c[i,j] = sum_{a<=i,b<=j} x[a,b] y[i-a,j-b]."""
    out = np.zeros(np.broadcast_shapes(x.shape, y.shape))
    for i in range(DEG_EPS + 1):
        for j in range(DEG_T + 1):
            acc = 0.0
            for a in range(i + 1):
                for b in range(j + 1):
                    acc = acc + x[a, b] * y[i - a, j - b]
            out[i, j] = acc
    return out


def tanh_derivatives(x0):
    """tanh and its first four derivatives at x0, from T' = 1 - T^2 applied
    repeatedly: T'' = -2 T s, T''' = -2 s (1 - 3 T^2), T'''' = 8 T s (2 - 3 T^2)
    with s = 1 - T^2."""
    T = np.tanh(x0)
    s = 1.0 - T * T
    return [T, s, -2.0 * T * s, -2.0 * s * (1.0 - 3.0 * T * T), 8.0 * T * s * (2.0 - 3.0 * T * T)]


def tanh(x):
    """tanh of a series by its Taylor expansion about the constant term:
    tanh(x00 + delta) = sum_k tanh^(k)(x00) / k! * delta^k.  delta has no
    constant term and total degree <= 4 survives truncation, so k <= 4."""
    x0 = x[0, 0]
    delta = x.copy()
    delta[0, 0] = 0.0
    ders = tanh_derivatives(x0)
    out = constant(ders[0])
    power = constant(np.ones_like(x0))
    for k in range(1, 5):
        power = mul(power, delta)
        out = out + (ders[k] / math.factorial(k)) * power
    return out


def affine(W, b, V, bv, h):
    """Linear layer with parameters moving along t:
    z = (W + t V) h + (b + t bv), with h a series of batch shape (..., in).
    W, V are [out, in]; b, bv are [out].  V/bv may be None (no t-motion)."""
    out = np.einsum("oi,ab...i->ab...o", W, h)
    out[0, 0] += b
    if V is not None:
        Vh = np.einsum("oi,ab...i->ab...o", V, h)
        out[:, 1:] += Vh[:, :-1]
        out[0, 1] += bv
    return out
