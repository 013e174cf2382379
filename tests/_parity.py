"""Error measures shared by the GPU parity tests (test infrastructure only).

* ``rel``: relative 2-norm error ||a - b|| / ||b||.
* ``elem``: the largest entry error relative to the entry plus the RMS of the
  reference, max_i |a_i - b_i| / (|b_i| + rms(b)).  An error spread over the
  entries at normwise level e gives a few e here (the largest of n roughly
  Gaussian entries is ~sqrt(2 ln n) times their RMS, 4-5 for n ~ 1e3-1e5),
  so ``check`` allows 10x the normwise tolerance; an error confined to a few
  small entries (one residual class, the biases, one layer) shows up in full
  (up to sqrt(n) times its normwise size) instead of being hidden by the
  large entries.
* ``blocks``: the error of each named block (each layer's W and b in the
  parameter layout; each residual class of an m-vector) relative to the
  block's norm plus the block's share of the RMS floor, ||a_B - b_B|| /
  (||b_B|| + rms(b) sqrt(|B|)).
"""
import numpy as np


def host(a):
    return a.detach().cpu().numpy() if hasattr(a, "detach") else np.asarray(a)


def rel(a, b):
    a = host(a)
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def elem(a, b):
    a = host(a)
    b = np.asarray(b)
    rms = float(np.sqrt(np.mean(b * b))) if b.size else 0.0
    if rms == 0.0:
        return float(np.max(np.abs(a - b))) if b.size else 0.0
    return float(np.max(np.abs(a - b) / (np.abs(b) + rms)))


def layer_blocks(widths):
    """(name, start, end) of W_l and b_l in the parameter vector."""
    out, off = [], 0
    for l in range(1, len(widths)):
        nw = widths[l] * widths[l - 1]
        out.append((f"W{l}", off, off + nw))
        out.append((f"b{l}", off + nw, off + nw + widths[l]))
        off += nw + widths[l]
    return out


def class_blocks(classes):
    out, off = [], 0
    for i, c in enumerate(classes):
        out.append((f"class{i}", off, off + int(c["count"])))
        off += int(c["count"])
    return out


def blocks(a, b, spans):
    a = host(a)
    b = np.asarray(b)
    rms = float(np.sqrt(np.mean(b * b))) if b.size else 0.0
    out = {}
    for name, s, e in spans:
        if e <= s:
            continue
        den = float(np.linalg.norm(b[s:e])) + rms * np.sqrt(e - s)
        out[name] = float(np.linalg.norm(a[s:e] - b[s:e]) / (den if den > 0 else 1.0))
    return out


def check(name, a, b, tol, spans=None, elem_tol=None):
    """Normwise and (optionally) blockwise errors of a against the reference
    b within tol, the entrywise one within elem_tol (default 10 tol)."""
    e_n = rel(a, b)
    e_e = elem(a, b)
    assert e_n <= tol, (name, "normwise", e_n, tol)
    assert e_e <= (10.0 * tol if elem_tol is None else elem_tol), (name, "entrywise", e_e, tol)
    if spans:
        bl = blocks(a, b, spans)
        worst = max(bl.values())
        assert worst <= tol, (name, "blockwise", bl)
    return e_n, e_e
