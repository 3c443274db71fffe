"""ctypes face of ``hsvd_oracle.c`` (test infrastructure only).

Every function here only moves numpy arrays in and out of the C oracle; the
arithmetic lives in ``hsvd_oracle.c`` and is described there with the paper's
section, equation or algorithm it follows.  The shared object is compiled with
gcc on first use (or by :func:`build`) into ``oracle/_build``.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

ORC_OK = 0
ORC_NOT_CONVERGED = 1
ORC_ARG = -1
ORC_RANK = -2
ORC_NONFINITE = -3

# how the iteration ended: not at all, a sweep without rotations (Eq. 2.3),
# every tangent of a sweep at most the threshold (Sec. 2, Eq. 4.2)
ORC_STOP_NONE = 0
ORC_STOP_ORTHO = 1
ORC_STOP_TANGENT = 2

# the paper's threshold T_eps = sqrt(eps) / 2 with eps = 2^-52, the smallest
# power of two with fl(1 + eps) > 1 (Sec. 2)
T_EPS = 2.0 ** -27

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hsvd_oracle.c")
# the exact model of the library's inner-solve kernels (not the oracle) is
# compiled into the same shared object; see inner_model.c and inner_model.py
_MODEL_SRC = os.path.join(_HERE, "inner_model.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liboracle_hsvd.so")
_lock = threading.Lock()
_lib = None

# optimisation without floating-point contraction: every fused multiply-add in
# the oracle is one written as fma(); -fopenmp is added when gcc has it
CFLAGS = ["-O2", "-ffp-contract=off"]

_p = ctypes.c_void_p
_i64 = ctypes.c_int64
_int = ctypes.c_int
_dbl = ctypes.c_double


def build(force=False, src=None, out=None):
    """Compile the oracle with gcc (-O2, no floating-point contraction).

    ``src``/``out`` compile another copy of the source (used by the tests
    that plant mistakes in a copy of the oracle)."""
    srcs = [_SRC, _MODEL_SRC] if src is None else [src]
    out = _SO if out is None else out
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if not force and os.path.exists(out) and all(os.path.getmtime(out) >= os.path.getmtime(f) for f in srcs):
        return out
    tmp = out + ".tmp.%d" % os.getpid()
    cmd = ["gcc"] + CFLAGS + ["-fPIC", "-shared", "-Wall", "-o", tmp] + srcs + ["-lm"]
    # the modulus order runs its steps' pairs on OpenMP threads when the
    # compiler has OpenMP; otherwise the same code is compiled serially
    if subprocess.run(cmd[:1] + ["-fopenmp"] + cmd[1:], capture_output=True).returncode != 0:
        subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


def _bind(lib):
    lib.orc_rotation.argtypes = [_dbl, _dbl, _dbl, _int, ctypes.POINTER(_dbl), ctypes.POINTER(_dbl)]
    lib.orc_rotation.restype = _int
    lib.orc_modulus_pairs.argtypes = [_int, _int, _p]
    lib.orc_modulus_pairs.restype = None
    lib.orc_hsvd.argtypes = [_i64, _i64, _p, _i64, _p, _dbl, _int, _int, _int,
                             _p, _p, _i64, _p, _i64, _p, _p, _dbl, _p]
    lib.orc_hsvd.restype = _int
    lib.orc_inner_solve.argtypes = [_int, _p, _p, _dbl, _int, _int, _int, _p, _p, _p, _p]
    lib.orc_set_threads.argtypes = [_int]
    lib.orc_set_threads.restype = _int
    lib.orc_inner_solve.restype = _int
    lib.orc_block_hsvd.argtypes = [_i64, _i64, _p, _i64, _p, _int, _dbl, _int, _int, _int,
                                   _int, _int, _p, _p, _i64, _p, _i64, _p, _p, _dbl, _p]
    lib.orc_block_hsvd.restype = _int
    lib.orc_sym_factor.argtypes = [_i64, _p, _i64, _p, _i64, _p, _p, _p]
    lib.orc_sym_factor.restype = _int
    lib.orc_hyp_qr.argtypes = [_i64, _i64, _p, _i64, _p, _p, _i64, _p, _p, _p, _i64, _p, _p, _p]
    lib.orc_hyp_qr.restype = _int
    lib.orc_hyp_qr_apply_tt.argtypes = [_i64, _i64, _p, _i64, _p, _p, _p, _p, _i64, _i64]
    lib.orc_hyp_qr_apply_tt.restype = _int
    lib.orc_wide_hsvd.argtypes = [_i64, _i64, _p, _i64, _p, _dbl, _int, _int, _p, _p, _i64, _p, _i64, _p, _p]
    lib.orc_wide_hsvd.restype = _int
    return lib


def load(path=None):
    """The oracle's shared object; ``path`` loads another build of the same
    source (the tests use this to run the pins against planted mistakes)."""
    global _lib
    if path is not None:
        return _bind(ctypes.CDLL(path))
    with _lock:
        if _lib is None:
            _lib = _bind(ctypes.CDLL(build()))
    return _lib


def _load():
    return load()


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def _fcol(G):
    return np.asfortranarray(np.asarray(G, dtype=np.float64))


def _signs(J, n):
    j = np.ascontiguousarray(np.asarray(J).astype(np.int8))
    if j.shape != (n,):
        raise ValueError("J must have one entry per column")
    return j


def rotation(aii, ajj, aij, hyp, lib=None):
    """(t, c, status) of the rotation annihilating a_ij (Sec. 2, Eq. 2.2)."""
    t, c = _dbl(), _dbl()
    st = (lib or _load()).orc_rotation(float(aii), float(ajj), float(aij), int(hyp), ctypes.byref(t), ctypes.byref(c))
    return t.value, c.value, st


def modulus_pairs(r, nsteps=None, lib=None):
    """Pivot pairs of the modified modulus strategy, shape (nsteps, r/2, 2)."""
    nsteps = r if nsteps is None else nsteps
    out = np.zeros((nsteps, r // 2, 2), dtype=np.int32)
    (lib or _load()).orc_modulus_pairs(int(r), int(nsteps), _ptr(out))
    return out


def set_threads(n=0, lib=None):
    """Threads of the modulus-parallel order (0: the OpenMP default); returns
    the count in use (1 for a build without OpenMP)."""
    return (lib or _load()).orc_set_threads(int(n))


def hsvd(G, J, tol, max_sweeps=30, order="cyclic", sort=False, want_u=True, want_v=True, lib=None, tstop=0.0):
    """Pointwise one-sided hyperbolic Jacobi SVD on the CPU.

    ``order`` is ``"cyclic"`` (row-cyclic) or ``"modulus"``.  ``tstop`` > 0
    also stops after a sweep whose tangents are all at most ``tstop`` (Sec. 2;
    ``T_EPS`` is the paper's value).  Returns a dict with sigma, U, V (input
    column order), sweeps, rotations, status and stop (ORC_STOP_*).
    """
    G = _fcol(G)
    m, n = G.shape
    j = _signs(J, n)
    sigma = np.zeros(n)
    U = np.zeros((m, n), order="F") if want_u else None
    V = np.zeros((n, n), order="F") if want_v else None
    sweeps, rots, stop = _int(), _i64(), _int()
    st = (lib or _load()).orc_hsvd(m, n, _ptr(G), m, _ptr(j), float(tol), int(max_sweeps),
                          1 if order == "modulus" else 0, 1 if sort else 0,
                          _ptr(sigma), _ptr(U), m, _ptr(V), n, ctypes.byref(sweeps), ctypes.byref(rots),
                          float(tstop), ctypes.byref(stop))
    return dict(sigma=sigma, U=U, V=V, sweeps=sweeps.value, rotations=rots.value, status=st, stop=stop.value)


_ORDERS = {"cyclic": 0, "parallel": 1}


def inner_solve(A, sgn, tol, mode=0, max_passes=8, order="cyclic", lib=None, want_tmax=False):
    """J-orthogonalise one pivot block, one rotation at a time; ``order`` is
    ``"cyclic"`` (row-cyclic, Sec. 5) or ``"parallel"`` (the pairs of the
    parallel strategy).  Returns (A_out, W, rotations, passes, status), and
    the largest applied |t| after them with ``want_tmax``."""
    A = np.array(A, dtype=np.float64, order="F", copy=True)
    nn = A.shape[0]
    s = _signs(sgn, nn)
    W = np.zeros((nn, nn), order="F")
    nrot, passes, tmax = _i64(), _int(), _dbl()
    st = (lib or _load()).orc_inner_solve(nn, _ptr(A), _ptr(s), float(tol), int(mode), _ORDERS[order],
                                          int(max_passes), _ptr(W), ctypes.byref(nrot), ctypes.byref(passes),
                                          ctypes.byref(tmax))
    if want_tmax:
        return A, W, nrot.value, passes.value, st, tmax.value
    return A, W, nrot.value, passes.value, st


def block_hsvd(G, J, b, tol, max_sweeps=30, inner_mode=0, inner_max_passes=8, sort=True,
               want_u=True, want_v=True, lib=None, tstop=0.0, inner_order="cyclic"):
    """Blocked one-sided hyperbolic Jacobi SVD on the CPU (block width b);
    ``tstop`` as for :func:`hsvd`, over the inner rotations' tangents;
    ``inner_order`` as ``order`` of :func:`inner_solve`."""
    G = _fcol(G)
    m, n = G.shape
    j = _signs(J, n)
    sigma = np.zeros(n)
    U = np.zeros((m, n), order="F") if want_u else None
    V = np.zeros((n, n), order="F") if want_v else None
    sweeps, rots, stop = _int(), _i64(), _int()
    st = (lib or _load()).orc_block_hsvd(m, n, _ptr(G), m, _ptr(j), int(b), float(tol), int(max_sweeps),
                                int(inner_mode), int(inner_max_passes), _ORDERS[inner_order], 1 if sort else 0,
                                _ptr(sigma), _ptr(U), m, _ptr(V), n, ctypes.byref(sweeps), ctypes.byref(rots),
                                float(tstop), ctypes.byref(stop))
    return dict(sigma=sigma, U=U, V=V, sweeps=sweeps.value, rotations=rots.value, status=st, stop=stop.value)


def sym_factor(M, lib=None, want_rank=False):
    """(G, J, perm, status) with M = G J G^T (Bunch-Parlett pivoting) for a
    symmetric M; perm[i] is the original index at position i.  A singular M
    stops once the trailing matrix is zero: with ``want_rank`` the rank r is
    returned fifth, and G's columns and J's entries past r are zero."""
    M = np.asfortranarray(np.asarray(M, dtype=np.float64))
    n = M.shape[0]
    G = np.zeros((n, n), order="F")
    J = np.zeros(n, dtype=np.int8)
    perm = np.zeros(n, dtype=np.int32)
    rank = _int()
    st = (lib or _load()).orc_sym_factor(n, _ptr(M), n, _ptr(G), n, _ptr(J), _ptr(perm), ctypes.byref(rank))
    if want_rank:
        return G, J, perm, st, rank.value
    return G, J, perm, st


def hyp_qr(A, J, lib=None):
    """Hyperbolic QR of a tall A (n x m) with signature J (n): a dict with R
    (m x m, block upper triangular), Jh (n signs after the row interchanges),
    cperm (the original column at each position), the reflectors refl
    (n x m), beta, rswap, bsize (1, or 2 and 0 for a 2 x 2 pivot) and status.
    T A[:, cperm] = [R; 0] with T^T diag(Jh) T = diag(J)."""
    A = _fcol(A)
    n, m = A.shape
    j = _signs(J, n)
    R = np.zeros((m, m), order="F")
    Jh = np.zeros(n, dtype=np.int8)
    cperm = np.zeros(m, dtype=np.int32)
    refl = np.zeros((n, m), order="F")
    beta = np.zeros(m)
    rswap = np.zeros(m, dtype=np.int32)
    bsize = np.zeros(m, dtype=np.int32)
    st = (lib or _load()).orc_hyp_qr(n, m, _ptr(A), n, _ptr(j), _ptr(R), m, _ptr(Jh), _ptr(cperm), _ptr(refl), n,
                                     _ptr(beta), _ptr(rswap), _ptr(bsize))
    return dict(R=R, Jh=Jh, cperm=cperm, refl=refl, beta=beta, rswap=rswap, bsize=bsize, status=st)


def hyp_qr_apply_tt(qr, X, lib=None):
    """T^T X for the transformation T of a :func:`hyp_qr` result (X n x c)."""
    X = np.array(X, dtype=np.float64, order="F", copy=True)
    if X.ndim == 1:
        X = X.reshape(-1, 1, order="F")
    n, c = X.shape
    m = qr["R"].shape[0]
    st = (lib or _load()).orc_hyp_qr_apply_tt(n, m, _ptr(qr["refl"]), n, _ptr(qr["beta"]), _ptr(qr["rswap"]),
                                              _ptr(qr["Jh"]), _ptr(X), n, c)
    if st != ORC_OK:
        raise ValueError("orc_hyp_qr_apply_tt: status %d" % st)
    return X


def wide_hsvd(G, J, tol, max_sweeps=30, order="cyclic", want_u=True, want_v=True, lib=None):
    """HSVD of a wide factor G (m x n, m <= n) through the hyperbolic QR of
    G^T: a dict with sigma, U (m x m), V (n x m), Jout (the m signs of the
    result, lambda_j = sigma_j^2 Jout_j), sweeps and status."""
    G = _fcol(G)
    m, n = G.shape
    j = _signs(J, n)
    sigma = np.zeros(m)
    U = np.zeros((m, m), order="F") if want_u else None
    V = np.zeros((n, m), order="F") if want_v else None
    Jout = np.zeros(m, dtype=np.int8)
    sweeps = _int()
    st = (lib or _load()).orc_wide_hsvd(m, n, _ptr(G), m, _ptr(j), float(tol), int(max_sweeps),
                                        1 if order == "modulus" else 0, _ptr(sigma), _ptr(U), m, _ptr(V), n,
                                        _ptr(Jout), ctypes.byref(sweeps))
    return dict(sigma=sigma, U=U, V=V, Jout=Jout, sweeps=sweeps.value, status=st)
