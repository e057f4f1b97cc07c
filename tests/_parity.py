"""Comparison used by every GPU-vs-oracle parity check.

rel(got, ref) is the larger of
  * the relative l2 error ||got - ref|| / ||ref||, and
  * the largest element error relative to the largest reference element,
    max|got - ref| / (5 max|ref|),
so an assertion rel(...) < tol bounds both the norm-wise error and every
single element (a localised error in low-amplitude elements, such as the tails
of a packet, cannot hide under a small l2 norm).  The factor 5 allows for
rounding noise spread evenly over many elements: for N elements of comparable
size the ratio of the two measures is about sqrt(2 ln N), 5.5 at N = 4M.
"""
import numpy as np


def rel(got, ref) -> float:
    got = np.asarray(got)
    ref = np.asarray(ref)
    d = got - ref
    l2 = float(np.linalg.norm(d) / np.linalg.norm(ref))
    mx = float(np.abs(d).max() / (5.0 * np.abs(ref).max())) if d.size else 0.0
    return max(l2, mx)
