"""Thin Python binding of the C ABI in ``include/hsvd.h`` (ctypes).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of ``libhsvd.so``.  PyTorch provides device memory and streams.  The
library is loaded on first use; if it has not been built (``build_lib.build()``
or ``__graft_entry__.build()``) the call raises -- there is no fallback.

Matrices are column-major: an m x n matrix is a tensor of shape (m, n) with
strides (1, ld).  Inputs in another layout are copied into that layout.
"""
import ctypes
import os
import threading
from dataclasses import dataclass
from typing import Optional

import torch

HSVD_OK = 0
HSVD_NOT_CONVERGED = 1
HSVD_ERR_ARG = -1
HSVD_ERR_RANK = -2
HSVD_ERR_NONFINITE = -3
HSVD_ERR_CUDA = -4
HSVD_ERR_NOMEM = -5

HSVD_METHOD_AUTO = 0
HSVD_METHOD_POINTWISE = 1
HSVD_METHOD_BLOCKED = 2
HSVD_INNER_ORIENTED = 0
HSVD_INNER_FULL = 1
HSVD_PRECISION_FP64 = 0
HSVD_PRECISION_BF16X8 = 1
HSVD_TSTOP_PAPER = 2.0 ** -27  # T_eps = sqrt(2^-52) / 2 (Sec. 2)
HSVD_STOP_NONE = 0
HSVD_STOP_ORTHO = 1
HSVD_STOP_TANGENT = 2
HSVD_SCHEDULE_AUTO = 0
HSVD_SCHEDULE_STEPS = 1
HSVD_SCHEDULE_PAIRS = 2
HSVD_SHORTEN_AUTO = 0
HSVD_SHORTEN_NEVER = 1
HSVD_SHORTEN_ALWAYS = 2

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libhsvd.so")
_lock = threading.Lock()
_lib = None

_p = ctypes.c_void_p
_i64 = ctypes.c_int64
_int = ctypes.c_int
_dbl = ctypes.c_double


HSVD_MLP_FEATURES = 8
HSVD_MLP_PARAMS = 4801
HSVD_TRACE_FIELDS = 8


class HsvdOpts(ctypes.Structure):
    _fields_ = [("tol", _dbl), ("max_sweeps", _int), ("method", _int), ("block_w", _int),
                ("inner_mode", _int), ("inner_max_passes", _int), ("sort", _int), ("profile", _int),
                ("precision", _int), ("skip_model", _p), ("skip_tau", _dbl), ("trace_out", _p),
                ("trace_cap", _i64), ("tstop", _dbl), ("schedule", _int), ("shorten", _int), ("jout", _p),
                ("reserved", _int * 2)]


class HsvdInfo(ctypes.Structure):
    _fields_ = [("sweeps", _int), ("method", _int), ("block_w", _int), ("status", _int),
                ("rotations", _i64), ("pair_updates", _i64), ("kernel_launches", _i64),
                ("ms_gram", _dbl), ("ms_solve", _dbl), ("ms_update", _dbl), ("ms_other", _dbl),
                ("pair_visits", _i64), ("masked_sweeps", _int), ("judge_sweeps", _int), ("trace_rows", _i64),
                ("stop_rule", _int), ("shortened", _int), ("ms_host_graph", _dbl)]


class HsvdBatchOpts(ctypes.Structure):
    _fields_ = [("tol", _dbl), ("max_sweeps", _int), ("sort", _int), ("group_width", _int), ("use_graph", _int),
                ("tstop", _dbl), ("cta_threads", _int), ("reserved", _int)]


class HsvdBatchInfo(ctypes.Structure):
    _fields_ = [("grid", _int), ("tuned", _int), ("bucket_width", _int * 5), ("max_sweeps_run", _int),
                ("rotations", _i64), ("kernel_launches", _i64), ("resident", _i64 * 3), ("ms_kernel", _dbl),
                ("ms_tune", _dbl), ("tangent_stops", _i64), ("cta_threads", _int)]


class HsvdError(RuntimeError):
    def __init__(self, status):
        super().__init__("hsvd failed: %s (%d)" % (hsvd_status_string(status), status))
        self.status = status


def lib():
    """The loaded ``libhsvd.so`` (raises if it was not built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError("libhsvd.so is not built (%s); run paper_1008_1371_gb300.build_lib.build()"
                                   % LIB_PATH)
            L = ctypes.CDLL(LIB_PATH)
            L.hsvd_default_opts.argtypes = [ctypes.POINTER(HsvdOpts)]
            L.hsvd_default_opts.restype = None
            L.hsvd_status_string.argtypes = [_int]
            L.hsvd_status_string.restype = ctypes.c_char_p
            L.hsvd_solve.argtypes = [_p, _i64, _i64, _i64, _p, _dbl, _int, _p, _p, _i64, _p, _i64, _p, _p]
            L.hsvd_solve.restype = _int
            L.hsvd_solve_ex.argtypes = [_p, _i64, _i64, _i64, _p, _p, _p, _i64, _p, _i64,
                                        ctypes.POINTER(HsvdOpts), ctypes.POINTER(HsvdInfo), _p]
            L.hsvd_solve_ex.restype = _int
            L.hsvd_modulus_pairs.argtypes = [_int, _int, _p]
            L.hsvd_modulus_pairs.restype = _int
            L.hsvd_ring_table.argtypes = [_int, _p]
            L.hsvd_ring_table.restype = _int
            L.hsvd_diag_wait_timeout.argtypes = [_p]
            L.hsvd_diag_wait_timeout.restype = _int
            L.hsvd_sym_factor.argtypes = [_p, _i64, _i64, _p, _i64, _p, _p, _p]
            L.hsvd_sym_factor.restype = _int
            L.hsvd_sym_eig.argtypes = [_p, _i64, _i64, _p, _p, _i64, ctypes.POINTER(HsvdOpts),
                                       ctypes.POINTER(HsvdInfo), _p]
            L.hsvd_sym_eig.restype = _int
            L.hsvd_shorten_qr.argtypes = [_p, _i64, _i64, _i64, _p, _i64, _p, _i64, _p]
            L.hsvd_shorten_qr.restype = _int
            L.hsvd_pivot_gram.argtypes = [_p, _i64, _i64, _int, _int, _p, _p, _p]
            L.hsvd_pivot_gram.restype = _int
            L.hsvd_pivot_solve.argtypes = [_int, _int, _p, _p, _dbl, _int, _int, _p, _p, _p, _p]
            L.hsvd_pivot_solve.restype = _int
            L.hsvd_pivot_update.argtypes = [_p, _i64, _i64, _int, _int, _p, _p, _p, _p]
            L.hsvd_pivot_update.restype = _int
            L.hsvd_pivot_gram_x.argtypes = [_p, _i64, _i64, _int, _p, _p, _p]
            L.hsvd_pivot_gram_x.restype = _int
            L.hsvd_pivot_update_x.argtypes = [_p, _i64, _i64, _int, _p, _p, _p, _p, _p]
            L.hsvd_pivot_update_x.restype = _int
            L.hsvd_mlp_forward.argtypes = [_p, _p, _i64, _p, _p]
            L.hsvd_mlp_forward.restype = _int
            L.hsvd_mlp_grad.argtypes = [_p, _p, _p, _i64, _p, _p, _p]
            L.hsvd_mlp_grad.restype = _int
            L.hsvd_mlp_adam.argtypes = [_p, _p, _p, _p, _int, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                        ctypes.c_float, _p]
            L.hsvd_mlp_adam.restype = _int
            L.hsvd_default_batch_opts.argtypes = [ctypes.POINTER(HsvdBatchOpts)]
            L.hsvd_default_batch_opts.restype = None
            L.hsvd_solve_batched.argtypes = [_i64, _p, _p, _p, _p, _p, _dbl, _int, _p, _p, _p, _p, _p, _p]
            L.hsvd_solve_batched.restype = _int
            L.hsvd_solve_batched_ex.argtypes = [_i64, _p, _p, _p, _p, _p, _p, _p, _p, _p, _p,
                                                ctypes.POINTER(HsvdBatchOpts), ctypes.POINTER(HsvdBatchInfo), _p]
            L.hsvd_solve_batched_ex.restype = _int
            _lib = L
    return _lib


def hsvd_status_string(status):
    return lib().hsvd_status_string(int(status)).decode()


def _colmajor(X, dtype):
    """(m, n) tensor with strides (1, ld >= m), converting if needed."""
    if X.dtype != dtype:
        X = X.to(dtype)
    m, n = X.shape
    if X.stride(0) == 1 and (n == 1 or X.stride(1) >= max(m, 1)):
        return X
    return X.t().contiguous().t()


def _empty_colmajor(m, n, like):
    return torch.empty((n, m), dtype=torch.float64, device=like.device,
                       pin_memory=(like.device.type == "cpu" and like.is_pinned())).t()


def _stream_ptr(stream, device):
    if device.type != "cuda":
        return None
    s = stream if stream is not None else torch.cuda.current_stream(device)
    return ctypes.c_void_p(s.cuda_stream)


def _need(cond, msg):
    if not cond:
        raise ValueError(msg)


def _check_vec(t, n, dtype, device, name):
    """A 1-D tensor of n elements, unit stride, on `device`."""
    _need(isinstance(t, torch.Tensor) and t.dtype == dtype and t.device == device, "%s: %s tensor on %s expected"
          % (name, dtype, device))
    _need(t.dim() == 1 and t.numel() == n and (n <= 1 or t.stride(0) == 1),
          "%s: %d contiguous elements expected, got shape %s" % (name, n, tuple(t.shape)))


def _check_colmajor(t, rows, cols, device, name):
    """A float64 rows x cols tensor on `device` in column-major layout
    (unit row stride, column stride >= rows)."""
    _need(isinstance(t, torch.Tensor) and t.dtype == torch.float64 and t.device == device,
          "%s: float64 tensor on %s expected" % (name, device))
    _need(t.dim() == 2 and tuple(t.shape) == (rows, cols), "%s: shape (%d, %d) expected, got %s"
          % (name, rows, cols, tuple(t.shape)))
    _need((rows <= 1 or t.stride(0) == 1) and (cols <= 1 or t.stride(1) >= rows),
          "%s: column-major layout expected (strides (1, >= %d)), got %s" % (name, rows, t.stride()))


def _ld(t, rows):
    """Leading dimension of a column-major tensor for the C ABI."""
    return t.stride(1) if t.shape[1] > 1 else max(rows, 1)


def _check_pairs(col0, ncols, b, disjoint=False, name="col0"):
    """Block pairs: an integer (npairs, 2) tensor of first columns, each block
    of b columns inside the ncols columns of the matrix, the two blocks of a
    pair apart; with `disjoint` (the in-place updates, where pairs run side
    by side) no two blocks of the table overlap."""
    _need(col0.dim() == 2 and col0.shape[0] >= 1 and col0.shape[1] == 2,
          "%s: integer tensor of shape (npairs >= 1, 2) expected" % name)
    c = col0.detach().to("cpu", torch.int64)
    _need(int(c.min()) >= 0 and int(c.max()) + b <= ncols,
          "%s: blocks of %d columns must lie inside the %d columns" % (name, b, ncols))
    _need(bool(((c[:, 0] - c[:, 1]).abs() >= b).all()), "%s: the two blocks of a pair overlap" % name)
    if disjoint:
        starts = torch.sort(c.reshape(-1)).values
        _need(bool((starts[1:] - starts[:-1] >= b).all()), "%s: blocks of different pairs overlap" % name)


@dataclass
class HsvdResult:
    sigma: torch.Tensor
    U: Optional[torch.Tensor]
    V: Optional[torch.Tensor]
    sweeps: int
    status: int
    method: int = 0
    block_w: int = 0
    rotations: int = 0
    pair_updates: int = 0
    kernel_launches: int = 0
    ms_gram: float = 0.0
    ms_solve: float = 0.0
    ms_update: float = 0.0
    ms_other: float = 0.0
    pair_visits: int = 0
    masked_sweeps: int = 0
    judge_sweeps: int = 0
    trace_rows: int = 0
    stop_rule: int = HSVD_STOP_NONE
    shortened: int = 0
    jout: Optional[torch.Tensor] = None  # wide factor: the m signs of the result (lambda = sigma^2 jout)
    ms_host_graph: float = 0.0  # host time capturing and instantiating sweep graphs


HSVD_SORT_AUTO = -1


def make_opts(tol=0.0, max_sweeps=30, method=HSVD_METHOD_AUTO, block_w=0, inner_mode=HSVD_INNER_ORIENTED,
              inner_max_passes=8, sort=None, profile=False, precision=HSVD_PRECISION_FP64, skip_model=None,
              skip_tau=0.0, trace_out=None, tstop=0.0, schedule=HSVD_SCHEDULE_AUTO, shorten=HSVD_SHORTEN_AUTO):
    """Options record; ``sort=None`` lets the library choose (sorting for the
    pointwise method only).  ``tstop``: tangent threshold of the early stop
    (0 = off, negative = HSVD_TSTOP_PAPER).  ``skip_model``: a float32 tensor of
    HSVD_MLP_PARAMS values (the learned form); ``trace_out``: a CUDA float32
    tensor of shape (rows, 9) receiving training rows.  The caller keeps both
    tensors alive while the options are in use."""
    o = HsvdOpts()
    lib().hsvd_default_opts(ctypes.byref(o))
    o.tol = float(tol)
    o.max_sweeps = int(max_sweeps)
    o.method = int(method)
    o.block_w = int(block_w)
    o.inner_mode = int(inner_mode)
    o.inner_max_passes = int(inner_max_passes)
    o.sort = HSVD_SORT_AUTO if sort is None else (1 if sort else 0)
    o.profile = 1 if profile else 0
    o.precision = int(precision)
    if skip_model is not None:
        if skip_model.dtype != torch.float32 or skip_model.numel() != HSVD_MLP_PARAMS or not skip_model.is_contiguous():
            raise ValueError("skip_model: contiguous float32 tensor of %d values" % HSVD_MLP_PARAMS)
        o.skip_model = skip_model.data_ptr()
    o.skip_tau = float(skip_tau)
    if trace_out is not None:
        if trace_out.dtype != torch.float32 or trace_out.dim() != 2 or trace_out.shape[1] != HSVD_MLP_FEATURES + 1 \
                or not trace_out.is_contiguous() or trace_out.device.type != "cuda":
            raise ValueError("trace_out: contiguous CUDA float32 tensor of shape (rows, 9)")
        o.trace_out = trace_out.data_ptr()
        o.trace_cap = trace_out.shape[0]
    o.tstop = float(tstop)
    o.schedule = int(schedule)
    o.shorten = int(shorten)
    return o


def hsvd_solve_ex(G, J, opts=None, compute_u=True, compute_v=True, stream=None, check=True, out=None):
    """HSVD of one factor: G V = U diag(sigma), U^T U = I, V^T J V = J.

    ``G`` (m x n float64) and ``J`` (n signs) are both CUDA tensors or both
    CPU tensors (pinned memory makes the copies asynchronous).  ``opts`` is an
    :class:`HsvdOpts` (see :func:`make_opts`).  ``out`` may hold preallocated
    (sigma, U, V) tensors in column-major layout.  A wide factor (m < n) is
    shortened by the hyperbolic QR of G^T first: sigma has m entries, U is
    m x m, V is n x m with V^T J V = diag(jout), and the result's ``jout``
    holds the m signs (the eigenvalues of G J G^T are sigma^2 jout).  Returns
    an :class:`HsvdResult`; raises :class:`HsvdError` on a negative status
    when ``check``.
    """
    L = lib()
    Gc = _colmajor(G, torch.float64)
    m, n = Gc.shape
    r = min(m, n)  # values and singular vectors
    Jc = J.to(torch.int8).contiguous()
    if Jc.device != Gc.device:
        raise ValueError("G and J must be on the same device")
    _need(Jc.dim() == 1 and Jc.numel() == n, "J: one sign per column of G (%d) expected" % n)
    pin = Gc.device.type == "cpu" and Gc.is_pinned()
    if out is not None:
        sigma, U, V = out
        _check_vec(sigma, r, torch.float64, Gc.device, "sigma")
        if U is not None:
            _check_colmajor(U, m, r, Gc.device, "U")
        if V is not None:
            _check_colmajor(V, n, r, Gc.device, "V")
    else:
        sigma = torch.empty(r, dtype=torch.float64, device=Gc.device, pin_memory=pin)
        U = _empty_colmajor(m, r, Gc) if compute_u else None
        V = _empty_colmajor(n, r, Gc) if compute_v else None
    o = opts if opts is not None else make_opts()
    jout = None
    if m < n:
        o = HsvdOpts.from_buffer_copy(o)
        jout = torch.zeros(m, dtype=torch.int8, device=Gc.device, pin_memory=pin)
        o.jout = jout.data_ptr()
    info = HsvdInfo()
    st = L.hsvd_solve_ex(Gc.data_ptr(), m, n, Gc.stride(1) if n > 1 else m, Jc.data_ptr(), sigma.data_ptr(),
                         U.data_ptr() if U is not None else None, _ld(U, m) if U is not None else m,
                         V.data_ptr() if V is not None else None, _ld(V, n) if V is not None else n,
                         ctypes.byref(o), ctypes.byref(info), _stream_ptr(stream, Gc.device))
    if check and st < 0:
        raise HsvdError(st)
    return HsvdResult(sigma, U, V, info.sweeps, st, info.method, info.block_w, info.rotations, info.pair_updates,
                      info.kernel_launches, info.ms_gram, info.ms_solve, info.ms_update, info.ms_other,
                      info.pair_visits, info.masked_sweeps, info.judge_sweeps, info.trace_rows, info.stop_rule,
                      info.shortened, jout, info.ms_host_graph)


def hsvd_solve(G, J, tol=0.0, max_sweeps=30, compute_u=True, compute_v=True, stream=None, check=True):
    """``hsvd_solve`` of the C ABI: default options with the given tol and sweep cap."""
    return hsvd_solve_ex(G, J, make_opts(tol=tol, max_sweeps=max_sweeps), compute_u, compute_v, stream, check)


def hsvd_modulus_pairs(r, nsteps=None):
    """The library's modified modulus table: int32 array (nsteps, r/2, 2)."""
    import numpy as np

    nsteps = r if nsteps is None else nsteps
    out = np.zeros((nsteps, r // 2, 2), dtype=np.int32)
    st = lib().hsvd_modulus_pairs(int(r), int(nsteps), out.ctypes.data_as(ctypes.c_void_p))
    if st != HSVD_OK:
        raise HsvdError(st)
    return out


def hsvd_ring_table(b):
    """The full pass's ring of slots: int32 array (2b, b, 4) of
    (lo, hi, buf_lo | buf_hi << 8, lo_arrived) per step and slot."""
    import numpy as np

    out = np.zeros((2 * b, b, 4), dtype=np.int32)
    st = lib().hsvd_ring_table(int(b), out.ctypes.data_as(ctypes.c_void_p))
    if st != HSVD_OK:
        raise HsvdError(st)
    return out


def hsvd_sym_factor(M, stream=None, want_rank=False):
    """(G, J) with M = G J G^T for a symmetric CUDA float64 tensor M (n x n).
    A singular M of rank r gives zero columns and signs past r; with
    ``want_rank`` the rank is returned third."""
    L = lib()
    Mc = _colmajor(M, torch.float64)
    n = Mc.shape[0]
    _need(Mc.shape[1] == n, "M must be square")
    G = _empty_colmajor(n, n, Mc)
    J = torch.empty(n, dtype=torch.int8, device=Mc.device)
    rank = ctypes.c_int64(0)
    st = L.hsvd_sym_factor(Mc.data_ptr(), n, Mc.stride(1) if n > 1 else n, G.data_ptr(), G.stride(1) if n > 1 else n,
                           J.data_ptr(), ctypes.byref(rank), _stream_ptr(stream, Mc.device))
    if st != HSVD_OK:
        raise HsvdError(st)
    return (G, J, rank.value) if want_rank else (G, J)


def hsvd_sym_eig(M, opts=None, compute_u=True, stream=None):
    """(lambda, U, info) of M = U diag(lambda) U^T through M = G J G^T and the
    HSVD of G; M a symmetric CUDA float64 tensor."""
    L = lib()
    Mc = _colmajor(M, torch.float64)
    n = Mc.shape[0]
    _need(Mc.shape[1] == n, "M must be square")
    lam = torch.empty(n, dtype=torch.float64, device=Mc.device)
    U = _empty_colmajor(n, n, Mc) if compute_u else None
    info = HsvdInfo()
    o = opts if opts is not None else make_opts()
    st = L.hsvd_sym_eig(Mc.data_ptr(), n, Mc.stride(1) if n > 1 else n, lam.data_ptr(),
                        U.data_ptr() if U is not None else None, (U.stride(1) if n > 1 else n) if U is not None else n,
                        ctypes.byref(o), ctypes.byref(info), _stream_ptr(stream, Mc.device))
    if st < 0:
        raise HsvdError(st)
    return lam, U, info


def hsvd_shorten_qr(G, want_q=True, stream=None):
    """(R, Q) of the shortening QR of a CUDA float64 tensor G (m x n, m >= n);
    Q is None unless want_q."""
    L = lib()
    Gc = _colmajor(G, torch.float64)
    m, n = Gc.shape
    R = _empty_colmajor(n, n, Gc)
    Q = _empty_colmajor(m, n, Gc) if want_q else None
    st = L.hsvd_shorten_qr(Gc.data_ptr(), m, n, Gc.stride(1) if n > 1 else m, R.data_ptr(), R.stride(1) if n > 1 else n,
                           Q.data_ptr() if Q is not None else None, (Q.stride(1) if n > 1 else m) if Q is not None else m,
                           _stream_ptr(stream, Gc.device))
    if st != HSVD_OK:
        raise HsvdError(st)
    return R, Q


def hsvd_pivot_gram(G, b, col0, stream=None):
    """A_P blocks (npairs, 2b, 2b) of the block pairs whose first columns are
    col0 (int32 CUDA tensor of shape (npairs, 2)); G column-major on the GPU,
    rows a multiple of 64."""
    L = lib()
    Gc = _colmajor(G, torch.float64)
    rows = Gc.shape[0]
    _check_pairs(col0, Gc.shape[1], b)
    npairs = col0.shape[0]
    c0 = col0.to(torch.int32).contiguous()
    A = torch.empty((npairs, 2 * b, 2 * b), dtype=torch.float64, device=Gc.device)
    st = L.hsvd_pivot_gram(Gc.data_ptr(), rows, Gc.stride(1), int(b), npairs, c0.data_ptr(), A.data_ptr(),
                           _stream_ptr(stream, Gc.device))
    if st != HSVD_OK:
        raise HsvdError(st)
    # blocks are column-major: element (x, y) at x + y*2b -> tensor [k, y, x]
    return A.transpose(1, 2)


def hsvd_pivot_solve(A, sgn, tol, mode=1, max_passes=8, stream=None):
    """J-orthogonalise pivot blocks A (npairs, 2b, 2b); returns
    (A_out, W, rotations, status)."""
    L = lib()
    _need(A.dim() == 3 and A.shape[1] == A.shape[2] and A.shape[1] in (32, 64, 128) and A.shape[0] >= 1,
          "A: (npairs, 2b, 2b) with b = 16, 32 or 64 expected")
    npairs, nn, _ = A.shape
    _need(tuple(sgn.shape) == (npairs, nn), "sgn: shape (npairs, 2b) expected")
    Ab = A.transpose(1, 2).contiguous().clone()  # column-major blocks
    W = torch.empty_like(Ab)
    s = sgn.to(torch.int8).contiguous()
    rot = torch.zeros(npairs, dtype=torch.int32, device=A.device)
    status = torch.zeros(1, dtype=torch.int32, device=A.device)
    st = L.hsvd_pivot_solve(nn // 2, npairs, Ab.data_ptr(), s.data_ptr(), float(tol), int(mode), int(max_passes),
                            W.data_ptr(), rot.data_ptr(), status.data_ptr(), _stream_ptr(stream, A.device))
    if st != HSVD_OK:
        raise HsvdError(st)
    return Ab.transpose(1, 2), W.transpose(1, 2), rot, status


def hsvd_pivot_update(X, b, col0, W, rotated, stream=None):
    """In place: X[:, I|J] <- X[:, I|J] W_k for pairs with rotated[k] != 0."""
    L = lib()
    if not (X.stride(0) == 1):
        raise ValueError("X must be column-major")
    rows = X.shape[0]
    _check_pairs(col0, X.shape[1], b, disjoint=True)
    _need(tuple(W.shape) == (col0.shape[0], 2 * b, 2 * b), "W: shape (npairs, 2b, 2b) expected")
    _need(rotated.numel() == col0.shape[0], "rotated: one flag per pair expected")
    c0 = col0.to(torch.int32).contiguous()
    Wb = W.transpose(1, 2).contiguous()
    r = rotated.to(torch.int32).contiguous()
    st = L.hsvd_pivot_update(X.data_ptr(), rows, X.stride(1), int(b), c0.shape[0], c0.data_ptr(), Wb.data_ptr(),
                             r.data_ptr(), _stream_ptr(stream, X.device))
    if st != HSVD_OK:
        raise HsvdError(st)
    return X


def hsvd_pivot_gram_x(G, col0, stream=None):
    """Split-precision A_P blocks (npairs, 128, 128) of the block pairs (b = 64)."""
    L = lib()
    Gc = _colmajor(G, torch.float64)
    rows = Gc.shape[0]
    _check_pairs(col0, Gc.shape[1], 64)
    c0 = col0.to(torch.int32).contiguous()
    npairs = c0.shape[0]
    A = torch.empty((npairs, 128, 128), dtype=torch.float64, device=Gc.device)
    st = L.hsvd_pivot_gram_x(Gc.data_ptr(), rows, Gc.stride(1), npairs, c0.data_ptr(), A.data_ptr(),
                             _stream_ptr(stream, Gc.device))
    if st != HSVD_OK:
        raise HsvdError(st)
    return A.transpose(1, 2)


def hsvd_pivot_update_x(X, col0, W, rotated, dexp=None, stream=None):
    """In place, split precision: X[:, I|J] <- X[:, I|J] W_k (b = 64)."""
    L = lib()
    if not (X.stride(0) == 1):
        raise ValueError("X must be column-major")
    _check_pairs(col0, X.shape[1], 64, disjoint=True)
    npairs = col0.shape[0]
    _need(tuple(W.shape) == (npairs, 128, 128), "W: shape (npairs, 128, 128) expected")
    _need(rotated.numel() == npairs, "rotated: one flag per pair expected")
    _need(dexp is None or tuple(dexp.shape) == (npairs, 128), "dexp: shape (npairs, 128) expected")
    c0 = col0.to(torch.int32).contiguous()
    Wb = W.transpose(1, 2).contiguous()
    r = rotated.to(torch.int32).contiguous()
    d = dexp.to(torch.int32).contiguous() if dexp is not None else None
    st = L.hsvd_pivot_update_x(X.data_ptr(), X.shape[0], X.stride(1), c0.shape[0], c0.data_ptr(), Wb.data_ptr(),
                               r.data_ptr(), d.data_ptr() if d is not None else None, _stream_ptr(stream, X.device))
    if st != HSVD_OK:
        raise HsvdError(st)
    return X


@dataclass
class HsvdBatchResult:
    sigma: list
    U: Optional[list]
    V: Optional[list]
    sweeps: list
    status: list
    rc: int
    info: HsvdBatchInfo


def make_batch_opts(tol=0.0, max_sweeps=30, sort=True, group_width=0, use_graph=True, tstop=0.0, cta_threads=0):
    """Batched-form options; ``cta_threads`` 512 selects the kernel with 512
    threads a CTA (twice the registers a thread), 0 the default 1024."""
    o = HsvdBatchOpts()
    lib().hsvd_default_batch_opts(ctypes.byref(o))
    o.cta_threads = int(cta_threads)
    o.tol = float(tol)
    o.max_sweeps = int(max_sweeps)
    o.sort = 1 if sort else 0
    o.group_width = int(group_width)
    o.use_graph = 1 if use_graph else 0
    o.tstop = float(tstop)
    return o


def _ptr_array(ptrs):
    arr = (ctypes.c_void_p * max(len(ptrs), 1))()
    for i, q in enumerate(ptrs):
        arr[i] = q
    return arr


def hsvd_solve_batched(Gs, Js, opts=None, compute_u=True, compute_v=True, stream=None, check=True, out=None):
    """``hsvd_solve_batched_ex``: independent HSVDs of the factors ``Gs`` (a
    list of m_k x n_k float64 tensors, all CUDA or all CPU) with signatures
    ``Js``, in one persistent launch.  ``out`` may hold preallocated
    (sigmas, Us, Vs) lists (column-major, leading dimensions m_k and n_k).
    Returns an :class:`HsvdBatchResult`; raises :class:`HsvdError` on a
    negative status when ``check``."""
    L = lib()
    count = len(Gs)
    Gc = [_colmajor(G, torch.float64) for G in Gs]
    Jc = [J.to(torch.int8).contiguous() for J in Js]
    if len(Jc) != count:
        raise ValueError("one signature per factor")
    dev = Gc[0].device if count else torch.device("cpu")
    m = (ctypes.c_int64 * max(count, 1))(*[G.shape[0] for G in Gc])
    n = (ctypes.c_int64 * max(count, 1))(*[G.shape[1] for G in Gc])
    ld = (ctypes.c_int64 * max(count, 1))(*[(G.stride(1) if G.shape[1] > 1 else G.shape[0]) for G in Gc])
    pin = dev.type == "cpu" and count > 0 and Gc[0].is_pinned()
    for k, (G, J) in enumerate(zip(Gc, Jc)):
        _need(G.device == dev and J.device == dev, "factor %d: every G and J on %s expected" % (k, dev))
        _need(J.dim() == 1 and J.numel() == G.shape[1], "factor %d: one sign per column of G expected" % k)
    if out is not None:
        sig, Us, Vs = out
        _need(len(sig) == count and (Us is None or len(Us) == count) and (Vs is None or len(Vs) == count),
              "out: one sigma, U and V per factor expected")
        for k, G in enumerate(Gc):
            mk, nk = G.shape
            _check_vec(sig[k], nk, torch.float64, dev, "sigma[%d]" % k)
            # the batched ABI takes leading dimensions m_k and n_k
            if Us is not None:
                _check_colmajor(Us[k], mk, nk, dev, "U[%d]" % k)
                _need(nk <= 1 or Us[k].stride(1) == mk, "U[%d]: leading dimension %d expected" % (k, mk))
            if Vs is not None:
                _check_colmajor(Vs[k], nk, nk, dev, "V[%d]" % k)
                _need(nk <= 1 or Vs[k].stride(1) == nk, "V[%d]: leading dimension %d expected" % (k, nk))
    else:
        sig = [torch.empty(G.shape[1], dtype=torch.float64, device=dev, pin_memory=pin) for G in Gc]
        Us = [torch.empty((G.shape[1], G.shape[0]), dtype=torch.float64, device=dev, pin_memory=pin).t()
              for G in Gc] if compute_u else None
        Vs = [torch.empty((G.shape[1], G.shape[1]), dtype=torch.float64, device=dev, pin_memory=pin).t()
              for G in Gc] if compute_v else None
    sweeps = (ctypes.c_int * max(count, 1))()
    status = (ctypes.c_int * max(count, 1))()
    o = opts if opts is not None else make_batch_opts()
    info = HsvdBatchInfo()
    rc = L.hsvd_solve_batched_ex(count, _ptr_array([G.data_ptr() for G in Gc]), m, n, ld,
                                 _ptr_array([J.data_ptr() for J in Jc]), _ptr_array([x.data_ptr() for x in sig]),
                                 _ptr_array([x.data_ptr() for x in Us]) if Us is not None else None,
                                 _ptr_array([x.data_ptr() for x in Vs]) if Vs is not None else None,
                                 sweeps, status, ctypes.byref(o), ctypes.byref(info), _stream_ptr(stream, dev))
    if check and rc < 0:
        raise HsvdError(rc)
    return HsvdBatchResult(sig, Us, Vs, list(sweeps)[:count], list(status)[:count], rc, info)


def _f32_cuda(t, shape=None):
    if t.dtype != torch.float32 or t.device.type != "cuda" or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA float32 tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError("expected shape %s, got %s" % (shape, tuple(t.shape)))
    return t


def hsvd_mlp_forward(params, X, stream=None):
    """Logits of the learned-form network for the rows of X (n x 8)."""
    _f32_cuda(params, (HSVD_MLP_PARAMS,))
    _f32_cuda(X)
    _need(X.dim() == 2 and X.shape[1] == HSVD_MLP_FEATURES, "X: shape (n, %d) expected" % HSVD_MLP_FEATURES)
    n = X.shape[0]
    out = torch.empty(n, dtype=torch.float32, device=X.device)
    rc = lib().hsvd_mlp_forward(params.data_ptr(), X.data_ptr(), n, out.data_ptr(), _stream_ptr(stream, X.device))
    if rc != HSVD_OK:
        raise HsvdError(rc)
    return out


def hsvd_mlp_grad(params, X, y, stream=None):
    """(gradient, mean loss) of the mean binary cross-entropy with logits."""
    _f32_cuda(params, (HSVD_MLP_PARAMS,))
    _f32_cuda(X)
    _need(X.dim() == 2 and X.shape[1] == HSVD_MLP_FEATURES, "X: shape (n, %d) expected" % HSVD_MLP_FEATURES)
    _f32_cuda(y, (X.shape[0],))
    g = torch.empty(HSVD_MLP_PARAMS, dtype=torch.float32, device=X.device)
    loss = torch.empty(1, dtype=torch.float32, device=X.device)
    rc = lib().hsvd_mlp_grad(params.data_ptr(), X.data_ptr(), y.data_ptr(), X.shape[0], g.data_ptr(),
                             loss.data_ptr(), _stream_ptr(stream, X.device))
    if rc != HSVD_OK:
        raise HsvdError(rc)
    return g, loss


def hsvd_mlp_adam(params, m, v, grad, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    """One Adam step on params (in place), moments m and v (in place)."""
    for x in (params, m, v, grad):
        _f32_cuda(x, (HSVD_MLP_PARAMS,))
    rc = lib().hsvd_mlp_adam(params.data_ptr(), m.data_ptr(), v.data_ptr(), grad.data_ptr(), int(t), float(lr),
                             float(beta1), float(beta2), float(eps), _stream_ptr(stream, params.device))
    if rc != HSVD_OK:
        raise HsvdError(rc)
