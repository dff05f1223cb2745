"""Closeness measure of the GPU parity tests."""
import numpy as np


def rel(a, b):
    """The larger of the normwise relative difference ||a - b||_F / ||b||_F
    and the entrywise one max |a - b| / max |b| over the whole block.

    The second catches a few wrong entries (a wrong row, a dropped term in one
    column) that a normwise bound over a large block would let through.  A
    zero reference is compared in absolute terms."""
    a = np.asarray(a)
    b = np.asarray(b)
    if a.shape != b.shape:
        raise AssertionError(f"shape {a.shape} != {b.shape}")
    if a.size == 0:
        return 0.0
    d = a - b
    nb = np.linalg.norm(b)
    mb = np.max(np.abs(b))
    norm_rel = np.linalg.norm(d) / (nb if nb > 0 else 1.0)
    elem_rel = np.max(np.abs(d)) / (mb if mb > 0 else 1.0)
    return float(max(norm_rel, elem_rel))
