"""ctypes face of ``inner_model.c``: the exact CPU model of the library's
inner-solve kernels (test infrastructure only, and not the oracle).

The oracle's inner solve (:func:`oracle.inner_solve`) applies one rotation at
a time in the paper's row-cyclic order.  The library's cluster kernels apply
the disjoint pairs of each step of the parallel strategy at once and
alternate the two halves of R^T A R between steps; this model repeats those
operations in the same order, so the kernels can be compared with it bit for
bit.  The model itself is bounded against the oracle by the tests."""
import ctypes

import numpy as np

from .oracle import _dbl, _i64, _int, _load, _p, _ptr, _signs


def _bound(lib):
    f = lib.mdl_inner_solve
    if getattr(f, "_bound", False):
        return f
    f.argtypes = [_int, _p, _p, _dbl, _int, _int, _p, _p, _p, _p]
    f.restype = _int
    f._bound = True
    return f


def inner_solve(A, sgn, tol, mode=0, max_passes=8, lib=None, want_tmax=False):
    """The kernels' inner solve of one pivot block (mode 0 full passes until
    none rotates, 1 one cross pass, 2 one full pass).  Returns (A_out, W,
    rotations, passes, status), and the largest applied |t| with
    ``want_tmax``."""
    A = np.array(A, dtype=np.float64, order="F", copy=True)
    nn = A.shape[0]
    s = _signs(sgn, nn)
    W = np.zeros((nn, nn), order="F")
    nrot, passes, tmax = _i64(), _int(), _dbl()
    st = _bound(lib or _load())(nn, _ptr(A), _ptr(s), float(tol), int(mode), int(max_passes), _ptr(W),
                                ctypes.byref(nrot), ctypes.byref(passes), ctypes.byref(tmax))
    if want_tmax:
        return A, W, nrot.value, passes.value, st, tmax.value
    return A, W, nrot.value, passes.value, st


def rotation(aii, ajj, aij, hyp, lib=None):
    """The model's rotation of one pair that fails Eq. 2.3 (reading M5 of
    inner_model.c): (t, c, q = 1/c, status), status nonzero for a
    rank-deficient hyperbolic pair."""
    lib = lib or _load()
    f = lib.mdl_rotation
    if not getattr(f, "_bound", False):
        f.argtypes = [_dbl, _dbl, _dbl, _int, ctypes.POINTER(_dbl), ctypes.POINTER(_dbl), ctypes.POINTER(_dbl)]
        f.restype = _int
        f._bound = True
    t, c, q = _dbl(), _dbl(), _dbl()
    st = f(float(aii), float(ajj), float(aij), int(hyp), ctypes.byref(t), ctypes.byref(c), ctypes.byref(q))
    return t.value, c.value, q.value, st
