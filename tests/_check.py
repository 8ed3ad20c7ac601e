"""Comparison helpers shared by the parity tests.

Every parity check applies two bounds to an output matrix x against its
reference r (same shape):
  * relative Frobenius norm  ||x - r||_F / ||r||_F <= tol   (the error metric
    of the whole matrix, robust to the cancellations of Eq. (2bse) and of
    the two lines of Eq. (collint));
  * element-wise            max |x - r| <= tol * max |r|    (so that a small
    block of wrong entries cannot hide under a large norm).
"""
import numpy as np


def rel(a, b):
    """Relative Frobenius-norm error of a against b."""
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def elem(a, b):
    """Largest entry-wise error of a against b, relative to b's largest entry."""
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def check(a, b, tol, what=""):
    """Assert both bounds; returns the relative Frobenius error."""
    a = np.asarray(a)
    b = np.asarray(b)
    assert a.shape == b.shape, f"{what}: shape {a.shape} != {b.shape}"
    assert np.isfinite(a).all(), f"{what}: non-finite values"
    e, m = rel(a, b), elem(a, b)
    assert e <= tol and m <= tol, f"{what}: rel {e:.3e}, element-wise {m:.3e} (tol {tol:.1e})"
    return e
