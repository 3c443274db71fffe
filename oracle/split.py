"""Exact CPU models of the split-precision Gram and update (the BF16x8 form).

TEST INFRASTRUCTURE ONLY: the tests import it; the library never does, and
the two share no code.

Definition (the library's reading of the split scheme; Ozaki et al.'s error-
free splitting with balanced digits):

- A row window holds WINDOW = 512 consecutive rows of the 2b = 128 pivot-block
  columns.  Column c of the window gets E_c, the smallest E with |x| < 2^E
  for every normal entry x of it (0 when it has none); zero and subnormal
  entries count as 0.
- Each entry becomes the 55-bit integer V = trunc(x 2^(55 - E_c)) and its
  balanced base-128 digits: with W = V + B, B = 64 (128^7 - 1) / 127,
  q_1 = floor(W / 2^49) and q_k = (floor(W / 128^(8-k)) mod 128) - 64 for
  k = 2..8, so that V = sum_k q_k 128^(8-k).  Slice k is q_k 2^(1-7k).
- The window's (i, j) entry keeps the slice products with k + l <= 9,
  T = sum_rows sum_{k+l<=9} q_k(x_ri) q_l(x_rj) 2^(63-7(k+l)) (an exact
  integer), and is T 2^(E_i + E_j - 61) rounded once to the nearest double
  (ties to even).
- A_P is the sum of the windows' values in window order, in double
  precision, starting from 0.

The update [X_I X_J] <- [X_I X_J] W (X with 2b = 128 columns) balances the
columns first: with D = diag(2^dk_k), X W = (X D^-1)(D W).  Row i of X gets
E_i = max_k (e(x_ik) - dk_k) and column j of W gets F_j = max_k (e(w_kj) +
dk_k), e(x) the exponent with |x| < 2^e(x) (zero and subnormal entries do
not count; an empty maximum gives 0).  x_ik is split against E_i + dk_k and
w_kj against F_j - dk_k, the kept products (k + l <= 9) are summed exactly
over the 128 columns, and each output is that sum times 2^(E_i + F_j - 61)
rounded once.

The integer sums are formed with float64 matrix products: every digit
product is at most 64^2 and a sum of them stays below 2^24, so those
products are exact.
"""
from fractions import Fraction

import numpy as np

WINDOW = 512
SLICES = 8
MAX_D = 9
BIAS = 64 * sum(128 ** j for j in range(7))
TINY = 2.0 ** -1022  # smallest normal double


def column_exponents(P):
    """E_c for each column of P (rows x cols): |x| < 2^E_c over the normal
    entries, 0 for a column without one."""
    A = np.abs(np.asarray(P, dtype=np.float64))
    normal = A >= TINY
    _, e = np.frexp(np.where(normal, A, 1.0))
    e = np.where(normal, e.astype(np.int64), -(1 << 40))
    E = e.max(axis=0) if A.shape[0] else np.full(A.shape[1], -(1 << 40), dtype=np.int64)
    return np.where(E < -100000, 0, E).astype(np.int64)


def digits(P, E):
    """Balanced digits q[k-1] (k = 1..8) of every entry of P against the
    column exponents E; int64 arrays of P's shape."""
    P = np.asarray(P, dtype=np.float64)
    scaled = np.ldexp(np.where(np.abs(P) >= TINY, P, 0.0), (55 - np.asarray(E, dtype=np.int64))[None, :])
    V = np.trunc(scaled).astype(np.int64)  # |V| < 2^55: exact
    W = V + BIAS
    q = [W >> 49] + [((W >> (7 * (SLICES - k))) & 127) - 64 for k in range(2, SLICES + 1)]
    return np.stack(q)


def window_gram(P):
    """(value matrix, T matrix of Python ints, E) of one row window."""
    P = np.asarray(P, dtype=np.float64)
    E = column_exponents(P)
    q = digits(P, E).astype(np.float64)
    n = P.shape[1]
    Id = {}
    for d in range(2, MAX_D + 1):
        acc = np.zeros((n, n))
        for k in range(1, d):
            l = d - k
            if 1 <= l <= SLICES and k <= SLICES:
                acc += q[k - 1].T @ q[l - 1]
        Id[d] = acc
    T = [[0] * n for _ in range(n)]
    val = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            t = 0
            for d in range(2, MAX_D + 1):
                t += int(Id[d][i, j]) << (63 - 7 * d)
            T[i][j] = t
            val[i, j] = float(Fraction(t) * Fraction(2) ** int(E[i] + E[j] - 61))
    return val, T, E


def gram(P):
    """A_P of the pivot-block columns P (rows x 2b) as the split-precision
    Gram computes it: windows of WINDOW rows, summed in window order."""
    P = np.asarray(P, dtype=np.float64)
    rows, n = P.shape
    A = np.zeros((n, n))
    for r0 in range(0, max(rows, 1), WINDOW):
        val, _, _ = window_gram(P[r0:r0 + WINDOW])
        A = A + val
    return A


def _exponents(A):
    """e(x) for every entry (|x| < 2^e(x)); a large negative value for zero
    and subnormal entries."""
    A = np.abs(np.asarray(A, dtype=np.float64))
    normal = A >= TINY
    _, e = np.frexp(np.where(normal, A, 1.0))
    return np.where(normal, e.astype(np.int64), -(1 << 40))


def _digits_against(P, Eel):
    """Balanced digits of every entry of P split against the per-entry
    exponents Eel (same shape)."""
    P = np.asarray(P, dtype=np.float64)
    V = np.trunc(np.ldexp(np.where(np.abs(P) >= TINY, P, 0.0), 55 - Eel)).astype(np.int64)
    W = V + BIAS
    return np.stack([W >> 49] + [((W >> (7 * (SLICES - k))) & 127) - 64 for k in range(2, SLICES + 1)])


def _combine(qa, qb, escale):
    """sum over the shared index of the kept slice products of qa (8 x r x K)
    and qb (8 x K x c), times 2^(escale - 61) (escale r x c), rounded once."""
    r, c = qa.shape[1], qb.shape[2]
    Id = {}
    for d in range(2, MAX_D + 1):
        acc = np.zeros((r, c))
        for k in range(1, d):
            l = d - k
            if 1 <= l <= SLICES and k <= SLICES:
                acc += qa[k - 1] @ qb[l - 1]
        Id[d] = acc
    out = np.zeros((r, c))
    for i in range(r):
        for j in range(c):
            t = 0
            for d in range(2, MAX_D + 1):
                t += int(Id[d][i, j]) << (63 - 7 * d)
            out[i, j] = float(Fraction(t) * Fraction(2) ** int(escale[i, j] - 61))
    return out


def update(X, W, dk=None):
    """[X_I X_J] W as the split-precision update computes it: X (rows x 128)
    the panel, W (128 x 128) the pivot block's transformation, dk (128 ints)
    the balancing exponents (None: no balancing)."""
    X = np.asarray(X, dtype=np.float64)
    W = np.asarray(W, dtype=np.float64)
    n = W.shape[0]
    dk = np.zeros(n, dtype=np.int64) if dk is None else np.asarray(dk, dtype=np.int64)
    E = (_exponents(X) - dk[None, :]).max(axis=1) if n else np.zeros(X.shape[0], dtype=np.int64)
    E = np.where(E < -100000, 0, E)
    F = (_exponents(W) + dk[:, None]).max(axis=0)
    F = np.where(F < -100000, 0, F)
    qx = _digits_against(X, E[:, None] + dk[None, :]).astype(np.float64)
    qw = _digits_against(W, F[None, :] - dk[:, None]).astype(np.float64)
    return _combine(qx, qw, E[:, None] + F[None, :])
