"""Error measure of the GPU parity tests.

rel(a, b) is the error of a against the reference b: the larger of the
relative 2-norm error ||a - b|| / ||b|| and the element-wise error
max|a - b| / max|b|.  A bound on it therefore holds for the whole array and
for every single element on the array's own scale, so that one wrong value
(a pixel at a facet seam, a cell of a wrapped window, one visibility) cannot
hide in the norm of a large array.
"""
import numpy as np


def _as(x, cplx):
    x = np.asarray(x)
    return x.astype(np.complex128 if cplx else np.float64)


def rel(a, b):
    cplx = np.iscomplexobj(a) or np.iscomplexobj(b)
    a, b = _as(a, cplx), _as(b, cplx)
    a, b = np.broadcast_arrays(a, b)
    if b.size == 0:
        return 0.0
    d = a - b
    r2 = np.linalg.norm(d) / max(np.linalg.norm(b), 1e-300)
    ri = np.abs(d).max() / max(np.abs(b).max(), 1e-300)
    return float(max(r2, ri))


def rel2(a, b):
    """The relative 2-norm error alone (reported beside rel)."""
    cplx = np.iscomplexobj(a) or np.iscomplexobj(b)
    a, b = _as(a, cplx), _as(b, cplx)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
