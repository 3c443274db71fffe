"""Pins for the exact CPU models of the split-precision Gram and update (the
BF16x8 form: 55-bit truncation, balanced base-128 digits, the slice products
with k + l <= 9 summed exactly, one rounding), against what is fixed outside
them: exact rational
dot products (Python fractions), the digit identity V = sum q_k 128^(8-k),
inputs whose digits the kept products cover completely (then the model is
the exact dot product rounded once), the error bound of the dropped products
and the truncation, symmetry and power-of-two scaling.  CPU only."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import split

U = 2.0 ** -53


def _exact_dot(x, y):
    return sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(x, y))


def test_digits_reconstruct_the_truncated_integer():
    rng = np.random.default_rng(1)
    E = rng.integers(-30, 30, size=16)
    P = rng.uniform(-1, 1, size=(200, 16)) * np.exp2(E)[None, :]
    P[0] = np.nextafter(np.exp2(E), 0)  # just below 2^E
    P[1] = -P[0]
    assert np.array_equal(split.column_exponents(P), E)
    q = split.digits(P, E)
    assert q.shape == (8, 200, 16)
    assert q[0].min() >= -64 and q[0].max() <= 64 and q[1:].min() >= -64 and q[1:].max() <= 63
    for r in (0, 1, 7, 199):
        for c in (0, 5, 15):
            V = sum(int(q[k, r, c]) * 128 ** (7 - k) for k in range(8))
            want = int(Fraction(float(P[r, c])) * Fraction(2) ** int(55 - E[c]))  # truncation toward zero
            assert V == want, (r, c)


@pytest.mark.parametrize("rows", [1, 37, 512, 700])
def test_four_digit_inputs_are_exact(rows):
    """Entries n 2^(E-27), |n| < 2^27, have digits q_5..q_8 = 0, so every
    product has k + l <= 8 and is kept: each window's value is its exact dot
    product rounded once, and windows add in order."""
    rng = np.random.default_rng(rows)
    n = 6
    E = rng.integers(-20, 20, size=n)
    N = rng.integers(-(2 ** 27) + 1, 2 ** 27, size=(rows, n))
    N[0] = 2 ** 26 + 1  # pins E_c = E
    P = N.astype(np.float64) * np.exp2(E - 27)[None, :]
    A = split.gram(P)
    for i in range(n):
        for j in range(n):
            acc = 0.0
            for r0 in range(0, rows, split.WINDOW):
                acc = acc + float(_exact_dot(P[r0:r0 + split.WINDOW, i], P[r0:r0 + split.WINDOW, j]))
            assert A[i, j] == acc, (i, j)


@pytest.mark.parametrize("rows,spread", [(64, 0.0), (512, 3.0), (900, 6.0)])
def test_error_bound(rows, spread):
    """Per row, the truncation costs at most 2 2^-55 and the dropped products
    (k + l >= 10) at most 3.53 2^-55 of 2^(E_i + E_j): a window of K rows is
    within 5.6 K 2^-55 2^(E_i + E_j) of the exact dot product, plus one
    rounding; the windows' sum adds one rounding per window."""
    rng = np.random.default_rng(int(rows + 10 * spread))
    n = 8
    P = rng.standard_normal((rows, n)) * 10.0 ** rng.uniform(-spread, spread, size=(rows, n))
    A = split.gram(P)
    for i in range(n):
        for j in range(i, n):
            exact = _exact_dot(P[:, i], P[:, j])
            bound = 0.0
            for r0 in range(0, rows, split.WINDOW):
                w = P[r0:r0 + split.WINDOW]
                E = split.column_exponents(w)
                part = abs(float(_exact_dot(w[:, i], w[:, j])))
                bound += 5.6 * w.shape[0] * 2.0 ** -55 * 2.0 ** int(E[i] + E[j]) + 2 * U * part
            bound += 2 * U * abs(A[i, j])
            assert abs(Fraction(float(A[i, j])) - exact) <= Fraction(bound), (i, j)


def test_symmetric_scaled_and_zero_columns():
    rng = np.random.default_rng(4)
    P = rng.standard_normal((300, 10))
    P[:, 3] = 0.0
    P[5, 7] = 1e-310  # a subnormal entry counts as zero
    A = split.gram(P)
    assert np.array_equal(A, A.T)
    assert np.all(A[3] == 0.0) and np.all(A[:, 3] == 0.0)
    Q = P.copy()
    Q[:, 2] *= 2.0 ** 40
    Q[:, 6] *= 2.0 ** -33
    B = split.gram(Q)
    s = np.ones(10)
    s[2], s[6] = 2.0 ** 40, 2.0 ** -33
    assert np.array_equal(B, A * s[:, None] * s[None, :])
    P2 = P.copy()
    P2[5, 7] = 0.0
    assert np.array_equal(split.gram(P2), A)


def _pinned(rng, shape, exps, axis):
    """Integers n 2^(e - 27), |n| < 2^27 (four base-128 digits), with one
    entry per row (axis 1) or column (axis 0) at (2^26 + 1) 2^(e - 27), so the
    split exponent is e there."""
    N = rng.integers(-(2 ** 27) + 1, 2 ** 27, size=shape)
    if axis == 1:
        N[:, 0] = 2 ** 26 + 1
        return N.astype(np.float64) * np.exp2(np.asarray(exps) - 27)[:, None]
    N[0, :] = 2 ** 26 + 1
    return N.astype(np.float64) * np.exp2(np.asarray(exps) - 27)[None, :]


def test_update_four_digit_inputs_are_exact():
    """Update without balancing on four-digit inputs: every kept product
    covers them, so each output is the exact dot product rounded once."""
    rng = np.random.default_rng(11)
    X = _pinned(rng, (20, 128), rng.integers(-10, 10, size=20), axis=1)
    Wm = _pinned(rng, (128, 128), rng.integers(-10, 10, size=128), axis=0)
    O = split.update(X, Wm)
    for i in (0, 7, 19):
        for j in (0, 1, 64, 127):
            assert O[i, j] == float(_exact_dot(X[i], Wm[:, j])), (i, j)


def test_update_balancing_shift_and_scaling():
    """A common shift of all dk moves E_i and F_j in opposite directions and
    changes no digit: the same bits.  A power of two on a row of X or a
    column of W scales that output row or column exactly."""
    rng = np.random.default_rng(12)
    X = rng.standard_normal((30, 128)) * 10.0 ** rng.uniform(-6, 0, 128)[None, :]
    Wm = np.eye(128) + 0.3 * rng.standard_normal((128, 128))
    dk = np.floor(np.log2(np.linalg.norm(X, axis=0))).astype(np.int64)
    O = split.update(X, Wm, dk)
    assert np.array_equal(split.update(X, Wm, dk + 5), O)
    X2 = X.copy()
    X2[3] *= 2.0 ** 30
    W2 = Wm.copy()
    W2[:, 9] *= 2.0 ** -20
    O2 = split.update(X2, W2, dk)
    ref = O.copy()
    ref[3] *= 2.0 ** 30
    ref[:, 9] *= 2.0 ** -20
    assert np.array_equal(O2, ref)


@pytest.mark.parametrize("balanced", [False, True])
def test_update_error_bound(balanced):
    """Against exact rational dot products: within 5.6 K 2^-55 of the scale
    2^(E_i + F_j) <= 4 max_k |x_ik 2^-dk_k| max_k |w_kj 2^dk_k|, plus one
    rounding.  Balancing a graded panel shrinks that scale for the small
    columns' outputs."""
    rng = np.random.default_rng(13 + balanced)
    X = rng.standard_normal((12, 128)) * 10.0 ** rng.uniform(-6, 0, 128)[None, :]
    Wm = np.eye(128) + 0.3 * rng.standard_normal((128, 128))
    Wm[:, 7] *= 1e-9
    dk = np.floor(np.log2(np.linalg.norm(X, axis=0))).astype(np.int64) if balanced else np.zeros(128, np.int64)
    O = split.update(X, Wm, dk)
    sx = np.max(np.abs(X) * np.exp2(-dk)[None, :], axis=1)
    sw = np.max(np.abs(Wm) * np.exp2(dk)[:, None], axis=0)
    for i in range(0, 12, 3):
        for j in (0, 7, 50, 127):
            exact = _exact_dot(X[i], Wm[:, j])
            bound = 5.6 * 128 * 2.0 ** -55 * 4 * sx[i] * sw[j] + U * abs(O[i, j])
            assert abs(Fraction(float(O[i, j])) - exact) <= Fraction(bound), (i, j)


@pytest.mark.parametrize("name,attr,value", [("drops_d9", "MAX_D", 8), ("wrong_bias", "BIAS", 63 * sum(
    128 ** j for j in range(7)))])
def test_pins_catch_planted_mistakes(monkeypatch, name, attr, value):
    monkeypatch.setattr(split, attr, value)
    caught = False
    for test in (test_digits_reconstruct_the_truncated_integer, lambda: test_error_bound(512, 3.0),
                 lambda: test_update_error_bound(True)):
        try:
            test()
        except AssertionError:
            caught = True
    assert caught, name
