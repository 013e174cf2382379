"""Flat parameter layout of the tanh MLP ansatz u_theta (Sec. 2.1, Sec. 5).

Layout (one convention shared by every consumer of theta): for each layer
l = 1..L+1 in order, the weight matrix W_l of shape [w_l, w_{l-1}] flattened
row-major, followed by the bias b_l of length w_l.  Hidden layers are followed
by tanh, the last (output) layer is affine.

Pins: the parameter counts the paper prints for its architectures
(Sec. 5.1-5.7, App. A.3) are reproduced by ``n_params``.
"""
import numpy as np


def n_params(widths):
    """Number of trainable parameters of an MLP with layer widths ``widths``
    (input width first, output width last)."""
    return int(sum(widths[l] * widths[l - 1] + widths[l] for l in range(1, len(widths))))


def layer_offsets(widths):
    """Offsets into theta: list of (w_offset, b_offset, out, in) per layer."""
    out, off = [], 0
    for l in range(1, len(widths)):
        o, i = widths[l], widths[l - 1]
        out.append((off, off + o * i, o, i))
        off += o * i + o
    return out


def unpack(theta, widths):
    """Split flat theta into [(W_l, b_l)] views (W_l is [out, in])."""
    theta = np.asarray(theta, dtype=np.float64)
    assert theta.shape == (n_params(widths),)
    layers = []
    for (wo, bo, o, i) in layer_offsets(widths):
        layers.append((theta[wo:wo + o * i].reshape(o, i), theta[bo:bo + o]))
    return layers


def pack(layers):
    """Inverse of ``unpack``."""
    parts = []
    for W, b in layers:
        parts.append(np.asarray(W, dtype=np.float64).ravel())
        parts.append(np.asarray(b, dtype=np.float64).ravel())
    return np.concatenate(parts)
