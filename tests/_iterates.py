"""Element-by-element comparison of V-cycle iterates with the oracle's.

An iterate passes when the largest pointwise difference over the whole grid
(ring included), divided by the largest |value| of the oracle's iterate, is
within the bound, and so is the relative L2 difference.  The pointwise test
catches a single wrong point (a boundary row, the edge of a coset) that a
norm over millions of points would hide.
"""

import numpy as np


def iterate_errors(got, want):
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    scale = max(float(np.abs(want).max()), 1e-300)
    elem = float(np.abs(got - want).max()) / scale
    l2 = float(np.linalg.norm(got - want)) / max(float(np.linalg.norm(want)), 1e-300)
    return elem, l2


def assert_iterate(got, want, tol, l2_tol=None, what=""):
    """max|got - want| / max|want| <= tol and ||got - want|| / ||want|| <= l2_tol (default tol)."""
    elem, l2 = iterate_errors(got, want)
    l2_tol = tol if l2_tol is None else l2_tol
    assert elem <= tol and l2 <= l2_tol, f"{what} pointwise {elem:.3e} (bar {tol:.1e}), L2 {l2:.3e} (bar {l2_tol:.1e})"
