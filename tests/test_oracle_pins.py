"""Pins for the CPU oracle: checks against what the paper and mathematics fix,
independent of the oracle's own code (closed forms in exact arithmetic, LAPACK
via numpy, high-precision brute force, constructed ground truth, the paper's
tables).  No GPU needed."""
import os
from fractions import Fraction

import mpmath
import numpy as np
import pytest

from paper_1008_1371_gb300 import workloads as W

U = 2.0 ** -53
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _tol(n):
    return n * U


# --------------------------------------------------------------------------
# Pin 1: the 2x2 rotation (Sec. 2, Eq. 2.2, Eq. 2.6, Alg. 4.5)
# --------------------------------------------------------------------------
def _random_pivots(rng, count):
    for _ in range(count):
        x = rng.standard_normal(5) * 10.0 ** rng.uniform(-4, 4)
        y = rng.standard_normal(5) * 10.0 ** rng.uniform(-4, 4)
        yield x, y


@pytest.mark.parametrize("hyp", [-1, 1])
def test_rotation_root_exact(orc, hyp):
    """t solves a_ij (1 + hyp t^2) + t (a_ii + hyp a_jj) = 0 (the condition
    a'_ij = 0 under the update of Alg. 4.5), checked in exact rational
    arithmetic on the returned double; and it is the smaller root."""
    rng = np.random.default_rng(11)
    for x, y in _random_pivots(rng, 400):
        aii, ajj, aij = float(x @ x), float(y @ y), float(x @ y)
        t, c, st = orc.rotation(aii, ajj, aij, hyp)
        assert st == 0
        assert abs(t) <= 1.0
        F = Fraction
        resid = F(aij) * (1 + hyp * F(t) ** 2) + F(t) * (F(aii) + hyp * F(ajj))
        scale = abs(F(aij)) * (1 + F(t) ** 2) + abs(F(t)) * (F(aii) + F(ajj))
        assert abs(resid) <= 8 * U * scale
        # c is the cosine / hyperbolic cosine belonging to t
        expect = 1.0 / np.sqrt(1.0 - hyp * t * t)
        assert abs(c - expect) <= 4 * U * expect


@pytest.mark.parametrize("hyp", [-1, 1])
def test_rotation_eq26_and_junitary(orc, hyp):
    """Rotating the actual columns (in 60-digit arithmetic) annihilates a_ij and
    changes the diagonal as Eq. 2.6 says; the 2x2 transformation is
    J-unitary; trigonometric keeps the trace, hyperbolic lowers it (Sec. 5)."""
    mpmath.mp.dps = 60
    rng = np.random.default_rng(12)
    J2 = np.diag([1.0, 1.0 if hyp < 0 else -1.0])
    for x, y in _random_pivots(rng, 100):
        aii, ajj, aij = float(x @ x), float(y @ y), float(x @ y)
        t, c, st = orc.rotation(aii, ajj, aij, hyp)
        assert st == 0
        X = [mpmath.mpf(float(v)) for v in x]
        Y = [mpmath.mpf(float(v)) for v in y]
        T, C = mpmath.mpf(t), mpmath.mpf(c)
        Xn = [(xi + hyp * T * yi) * C for xi, yi in zip(X, Y)]
        Yn = [(T * xi + yi) * C for xi, yi in zip(X, Y)]
        A = lambda p, q: mpmath.fsum(a * b for a, b in zip(p, q))  # noqa: E731
        a_ii, a_jj, a_ij = A(X, X), A(Y, Y), A(X, Y)
        n_ii, n_jj, n_ij = A(Xn, Xn), A(Yn, Yn), A(Xn, Yn)
        scale = mpmath.sqrt(a_ii * a_jj)
        assert abs(n_ij) <= 16 * U * scale
        assert abs(n_ii - (a_ii + hyp * T * a_ij)) <= 16 * U * (a_ii + abs(a_ij))
        assert abs(n_jj - (a_jj + T * a_ij)) <= 16 * U * (a_jj + abs(a_ij))
        if hyp < 0:
            assert abs((n_ii + n_jj) - (a_ii + a_jj)) <= 16 * U * (a_ii + a_jj)
        else:
            assert n_ii + n_jj < a_ii + a_jj
        R = c * np.array([[1.0, t], [hyp * t, 1.0]])
        assert np.max(np.abs(R.T @ J2 @ R - J2)) <= 8 * U * max(1.0, c * c)


def test_rotation_cosine_unbiased(orc):
    """c = 1/sqrt(1 - hyp t^2) to rounding and without bias: over rotations
    with t^2 between u and 2^-30 the mean of c^2 (1 - hyp t^2) - 1 (exact
    rational arithmetic on the returned doubles) is within 0.1 u of 0, each
    within 2 u.  Evaluated as two rounded operations, 1/sqrt(1 + t^2) leans
    up by about u on average here (checked below as well): over the ~10^5
    rotations a column takes at n = 4096 that bias scales every sigma up by
    about 1e-12."""
    rng = np.random.default_rng(21)
    F = Fraction
    ours, naive = [], []
    for k in range(3000):
        hyp = -1 if k % 2 == 0 else 1
        aii = 1.0 + rng.random()
        ajj = aii * (1.0 + 0.5 * rng.random()) if hyp < 0 else aii * rng.random()
        b = (ajj - aii) if hyp < 0 else -(aii + ajj)
        tau = 10.0 ** rng.uniform(-7.8, -4.5)
        aij = rng.choice([-1.0, 1.0]) * abs(b) * tau
        t, c, st = orc.rotation(aii, ajj, aij, hyp)
        assert st == 0
        if not U <= t * t <= 2.0 ** -30:
            continue
        x = 1 - hyp * F(t) ** 2
        ours.append(float(F(c) ** 2 * x - 1) / U)
        xn = 1.0 - hyp * t * t if hyp < 0 else (1.0 - t) * (1.0 + t)
        naive.append(float(F(1.0 / np.sqrt(xn)) ** 2 * x - 1) / U)
    ours, naive = np.array(ours), np.array(naive)
    assert len(ours) >= 2000
    assert np.max(np.abs(ours)) <= 2.0
    assert abs(ours.mean()) <= 0.1
    assert naive.mean() >= 0.5


def test_rotation_closed_form_values(orc):
    # a_ii = a_jj: trigonometric rotation by pi/4 exactly
    t, c, st = orc.rotation(1.0, 1.0, 0.5, -1)
    assert st == 0 and t == 1.0 and abs(c - np.sqrt(0.5)) <= U
    # a_ii = 2, a_jj = 1, a_ij = 1/2, hyperbolic: zeta = -3, t = -(3 - 2 sqrt 2)
    t, c, st = orc.rotation(2.0, 1.0, 0.5, 1)
    assert st == 0
    assert abs(t + (3.0 - 2.0 * np.sqrt(2.0))) <= 4 * U
    assert abs(c - 1.0 / np.sqrt(1.0 - t * t)) <= 4 * U
    # a_ii = 5/2, a_jj = 1, a_ij = 1, trigonometric: zeta = -3/4, t = -1/2
    t, c, st = orc.rotation(2.5, 1.0, 1.0, -1)
    assert st == 0 and t == -0.5 and abs(c - 2.0 / np.sqrt(5.0)) <= U
    # parallel columns of equal norm and opposite sign: no hyperbolic rotation
    t, c, st = orc.rotation(1.0, 1.0, 1.0, 1)
    assert st == orc.ORC_RANK


# --------------------------------------------------------------------------
# Pin 2: J = I is the ordinary SVD (Sec. 1) -- LAPACK through numpy
# --------------------------------------------------------------------------
@pytest.mark.parametrize("kind", ["gaussian", "graded"])
def test_identity_signature_is_svd(orc, kind):
    n = 96
    G, _ = W.gaussian(n, seed=21) if kind == "gaussian" else W.graded(n, decades=3, seed=22)
    J = np.ones(n, dtype=np.int8)
    r = orc.hsvd(G, J, _tol(n), 40)
    assert r["status"] == 0
    sv = np.linalg.svd(G, compute_uv=False)
    got = np.sort(r["sigma"])[::-1]
    # LAPACK's backward-stable bound: |sigma - sigma_lapack| <= c n u sigma_max
    assert np.max(np.abs(got - sv)) <= 4 * n * U * sv[0]


# --------------------------------------------------------------------------
# Pin 3: invariants G V = U Sigma, U^T U = I, V^T J V = J (Eq. 1.1, Eq. 2.1)
# --------------------------------------------------------------------------
def _invariants(G, J, r):
    n = G.shape[1]
    Jd = np.diag(J.astype(np.float64))
    U_, V, s = r["U"], r["V"], r["sigma"]
    orth = np.max(np.abs(U_.T @ U_ - np.eye(n)))
    junit = np.max(np.abs(V.T @ Jd @ V - Jd)) / max(1.0, np.max(np.abs(V)) ** 2)
    resid = np.max(np.linalg.norm(G @ V - U_ * s[None, :], axis=0)
                   / (np.linalg.norm(G) * np.linalg.norm(V, axis=0)))
    return orth, junit, resid


@pytest.mark.parametrize("order,sort", [("cyclic", False), ("modulus", False), ("modulus", True)])
def test_invariants_pointwise(orc, order, sort):
    G, J = W.gaussian(128, seed=1)
    r = orc.hsvd(G, J, _tol(128), 30, order=order, sort=sort)
    assert r["status"] == 0
    orth, junit, resid = _invariants(G, J, r)
    n = 128
    assert orth <= 1e-12 * n and junit <= 1e-12 * n and resid <= 1e-12 * n
    assert orth <= 1e-13 and junit <= 1e-12 and resid <= 1e-15


# --------------------------------------------------------------------------
# Pin 4: eigenvalues of M = G J G^T are diag(Sigma^2 J) (Sec. 1), by LAPACK's
# symmetric eigensolver; and the pencil view: eig(J G^T G) = Sigma^2 J.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("p", [0, 17, 64, 128])
def test_eigen_cross_check(orc, p):
    n = 128
    G, _ = W.gaussian(n, seed=31)
    J = W.signs_block(n, p)
    r = orc.hsvd(G, J, _tol(n), 30, order="modulus", sort=True)
    assert r["status"] == 0
    lam = np.sort(r["sigma"] ** 2 * J)
    M = (G * J[None, :].astype(float)) @ G.T
    ev = np.sort(np.linalg.eigvalsh(M))
    assert np.max(np.abs(lam - ev)) <= 8 * n * U * np.max(np.abs(ev))
    pen = np.sort(np.linalg.eigvals(J[:, None] * (G.T @ G)).real)
    assert np.max(np.abs(lam - pen)) <= 1e-10 * np.max(np.abs(pen))


# --------------------------------------------------------------------------
# Pin 5: brute force on tiny inputs -- the roots of det(J G^T G - lambda I) in
# 60-digit arithmetic are sigma_k^2 j_k.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n,seed", [(2, 1), (3, 2), (4, 3), (5, 4), (6, 5), (6, 6)])
def test_brute_force_tiny(orc, n, seed):
    mpmath.mp.dps = 60
    rng = np.random.default_rng(100 + seed)
    m = n + (seed % 3)
    G = np.asfortranarray(rng.standard_normal((m, n)))
    J = np.where(rng.random(n) < 0.5, 1, -1).astype(np.int8)
    r = orc.hsvd(G, J, _tol(n), 40)
    assert r["status"] == 0
    Gm = mpmath.matrix(G.tolist())
    Jm = mpmath.diag([int(v) for v in J])
    ev = mpmath.eig(Jm * Gm.T * Gm, left=False, right=False)
    lam_true = sorted(float(mpmath.re(e)) for e in ev)
    lam = np.sort(r["sigma"] ** 2 * J)
    assert np.allclose(lam, lam_true, rtol=1e-13, atol=0)


# --------------------------------------------------------------------------
# Pin 6: constructed ground truth G = Q |Lambda|^(1/2) K, K J-unitary
# (spectrum shaped as in Sec. 5, Table 5.2): sigma = sqrt|lambda|.
# --------------------------------------------------------------------------
@pytest.mark.parametrize("n,p", [(64, 32), (96, 10), (160, 80)])
def test_constructed_ground_truth(orc, n, p):
    G, J, sig = W.paper(n, p=p, seed=60 + n)
    r = orc.hsvd(G, J, _tol(n), 40, order="modulus", sort=True)
    assert r["status"] == 0
    for s in (1, -1):
        got = np.sort(r["sigma"][J == s])
        ref = np.sort(sig[J == s])
        assert np.max(np.abs(got - ref) / ref) <= 1e-12


def test_orthogonality_scale(orc):
    """d(U) = ||I - U^T U||_F reported from 1.11e-14 at the smallest order
    (n = 160, Sec. 5); the oracle stays within a decade of that when the test
    of Eq. 2.3 uses epsilon = 2^-52 (the smallest power of two with
    fl(1 + eps) > 1 under round-to-nearest)."""
    G, J, _ = W.paper(160, seed=160)
    r = orc.hsvd(G, J, 2.0 ** -52, 40, order="modulus", sort=True)
    assert r["status"] == 0
    dU = np.linalg.norm(np.eye(160) - r["U"].T @ r["U"])
    assert dU <= 1.11e-13


# --------------------------------------------------------------------------
# Pin 7: the modified modulus strategy (Sec. 2, Alg. 4.3/4.4, Appendix)
# --------------------------------------------------------------------------
@pytest.mark.parametrize("r", [2, 4, 6, 8, 10, 16, 32, 64])
def test_modulus_strategy_properties(orc, r):
    P = orc.modulus_pairs(r, r + 1)
    cover = {}
    for s in range(r):
        idx = P[s].ravel()
        assert sorted(idx.tolist()) == list(range(r))  # r/2 disjoint pairs
        for a, b in P[s]:
            key = (min(a, b), max(a, b))
            cover[key] = cover.get(key, 0) + 1
    assert set(cover) == {(i, j) for i in range(r) for j in range(i + 1, r)}
    for (i, j), cnt in cover.items():
        assert cnt == (2 if j - i == r // 2 else 1)
    # the next quasi-sweep starts on the antidiagonal with tasks reversed
    start = [tuple(sorted(p)) for p in P[0]]
    assert start == [(k, r - 1 - k) for k in range(r // 2)]
    assert [tuple(sorted(p)) for p in P[r]] == start[::-1]


def _read_golden(name):
    rows = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            k, rest = line.split(":")
            rows[int(k)] = rest.split()
    return rows


def test_modulus_matches_appendix_tables(orc):
    n = 8
    anti = {k: {tuple(int(v) for v in p.split(",")) for p in ps}
            for k, ps in _read_golden("antidiagonal_n8.txt").items()}
    # the table's own rule, for every one of its 2n-3 steps
    for k, pairs in anti.items():
        assert pairs == {(i, k + 2 - i) for i in range(1, n + 1) if i < k + 2 - i <= n}
    steps = _read_golden("modulus_from_antidiagonal_n8.txt")
    P = orc.modulus_pairs(n)
    for s, ks in steps.items():
        got = {(min(a, b) + 1, max(a, b) + 1) for a, b in P[s]}
        want = set().union(*(anti[int(k)] for k in ks))
        extra = got - want
        assert want <= got
        assert all(j - i == n // 2 for i, j in extra) and len(extra) <= 1


# --------------------------------------------------------------------------
# Pin 8: the inner pivot-block solve (Sec. 5 / Sec. 6).  Rotations one at a
# time as R^T A R, row-cyclic (Sec. 5) or in the parallel strategy's pairs.
# --------------------------------------------------------------------------
ORDERS = ("cyclic", "parallel")


def _pivot_block(nn, seed, rows=None, lo=-2):
    rng = np.random.default_rng(seed)
    Gp = rng.standard_normal((rows or 3 * nn, nn)) * (10.0 ** rng.uniform(lo, 0, nn))[None, :]
    return Gp.T @ Gp


def _congruence_checks(A, sg, Ao, Wp, passes=1):
    """What every inner solve must give, whatever its pair order: W is
    J-unitary (W^T J W = J), A_out is the congruence W^T A W, A_out stays
    symmetric, and the eigenvalues of J A are unchanged (J A_out =
    W^-1 (J A) W, a similarity), the last against LAPACK."""
    nn = A.shape[0]
    Jd = np.diag(sg.astype(float))
    wmax = max(1.0, np.max(np.abs(Wp)) ** 2)
    assert np.max(np.abs(Wp.T @ Jd @ Wp - Jd)) <= 8 * passes * nn * U * wmax
    scale = np.abs(Wp).T @ np.abs(A) @ np.abs(Wp)
    assert np.all(np.abs(Wp.T @ A @ Wp - Ao) <= 8 * passes * nn * U * scale)
    assert np.array_equal(Ao, Ao.T)
    ev_in = np.sort(np.linalg.eigvals(Jd @ A).real)
    ev_out = np.sort(np.linalg.eigvals(Jd @ Ao).real)
    assert np.allclose(ev_out, ev_in, rtol=1e-10, atol=0)


@pytest.mark.parametrize("order", ORDERS)
def test_inner_solve_2x2_is_rotation(orc, order):
    rng = np.random.default_rng(81)
    for hyp in (-1, 1):
        sg = np.array([1, 1 if hyp < 0 else -1], dtype=np.int8)
        x, y = rng.standard_normal(4), rng.standard_normal(4)
        A = np.array([[x @ x, x @ y], [x @ y, y @ y]])
        t, c, _ = orc.rotation(A[0, 0], A[1, 1], A[0, 1], hyp)
        for mode in (0, 1, 2):
            Ao, Wp, nrot, passes, st = orc.inner_solve(A, sg, 1e-15, mode=mode, max_passes=4, order=order)
            assert st == 0 and nrot == 1
            assert np.allclose(Wp, c * np.array([[1.0, t], [hyp * t, 1.0]]), rtol=0, atol=4 * U)
            assert Ao[0, 1] == 0.0 and Ao[1, 0] == 0.0


@pytest.mark.parametrize("order", ORDERS)
@pytest.mark.parametrize("p", [0, 5, 16, 32])
def test_inner_solve_full_block_diagonalises(orc, p, order):
    """Full-block mode: W^T A W = diag(A_out) with W J-unitary, so the
    eigenvalues of J A are J diag(A_out) (a similarity), checked by LAPACK."""
    nn = 32
    A = _pivot_block(nn, 90 + p, rows=200)
    sg = W.signs_block(nn, p)
    Ao, Wp, nrot, passes, st = orc.inner_solve(A, sg, _tol(nn), mode=0, max_passes=20, order=order)
    assert st == 0 and passes < 20
    _congruence_checks(A, sg, Ao, Wp, passes)
    D = np.sqrt(np.diag(Ao))
    off = Ao - np.diag(np.diag(Ao))
    assert np.max(np.abs(off) / np.outer(D, D)) <= _tol(nn)
    ev = np.sort(np.linalg.eigvals(np.diag(sg.astype(float)) @ A).real)
    assert np.allclose(np.sort(sg * np.diag(Ao)), ev, rtol=1e-10, atol=0)


def test_inner_solve_full_block_orders_agree(orc):
    """Both pair orders diagonalise the same block to the same pencil
    eigenvalues (each sign group sorted)."""
    nn = 48
    A = _pivot_block(nn, 97)
    sg = W.signs_random(np.random.default_rng(3), nn, 20)
    d = [orc.inner_solve(A, sg, _tol(nn), mode=0, max_passes=20, order=o)[0] for o in ORDERS]
    for s in (1, -1):
        a, b = np.sort(np.diag(d[0])[sg == s]), np.sort(np.diag(d[1])[sg == s])
        assert np.allclose(a, b, rtol=1e-11, atol=0)


def _hand_block(hyp):
    """4 x 4 pivot block with two disjoint couplings, (0, 2) and (1, 3), and
    its cross pass worked by hand.  Trigonometric (J = I): a_00 = a_22 = 2,
    a_02 = 1, so zeta = 0, t = 1, c = 1/sqrt 2, the new diagonal 2 -+ 1 (Eq.
    2.6).  Hyperbolic (J = diag(1, 1, -1, -1)): a_00 = a_22 = 5, a_02 = -4,
    so zeta = 10/8, t = 1/(5/4 + 3/4) = 1/2, c = 1/sqrt(3/4), the new
    diagonal 5 + t a_02 = 3 twice (J A has eigenvalues +-3).  The pair (0, 3)
    and (1, 2) entries stay exactly zero, so the pass rotates two pairs."""
    if hyp < 0:
        a, b, sg, t, c, dp, dq = 2.0, 1.0, np.ones(4, dtype=np.int8), 1.0, 1 / np.sqrt(2.0), 1.0, 3.0
    else:
        a, b, sg, t, c, dp, dq = 5.0, -4.0, np.array([1, 1, -1, -1], dtype=np.int8), 0.5, 2 / np.sqrt(3.0), 3.0, 3.0
    A = np.array([[a, 0, b, 0], [0, a, 0, b], [b, 0, a, 0], [0, b, 0, a]], dtype=float)
    Wk = np.zeros((4, 4))
    for p, q in ((0, 2), (1, 3)):
        Wk[p, p], Wk[q, p] = c, hyp * t * c  # column p: (e_p + hyp t e_q) c
        Wk[p, q], Wk[q, q] = t * c, c  # column q: (t e_p + e_q) c
    return A, sg, Wk, np.diag([dp, dp, dq, dq])


@pytest.mark.parametrize("order", ORDERS)
@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("hyp", [-1, 1])
def test_inner_solve_hand_worked_block(orc, mode, hyp, order):
    A, sg, Wk, Dk = _hand_block(hyp)
    Ao, Wp, nrot, passes, st = orc.inner_solve(A, sg, _tol(4), mode=mode, order=order)
    assert st == 0 and nrot == 2 and passes == 1
    assert np.max(np.abs(Wp - Wk)) <= 4 * U * np.max(np.abs(Wk))
    assert np.max(np.abs(Ao - Dk)) <= 8 * U * np.max(np.abs(A))


@pytest.mark.parametrize("order", ORDERS)
@pytest.mark.parametrize("p", [0, 3, 8, 16])
def test_inner_solve_cross_pass(orc, order, p):
    """Cross pass (mode 1): a congruence by a J-unitary W that keeps J A's
    eigenvalues (LAPACK), rotating only pairs of the off-diagonal block: at
    most h^2 of them, and none at all when that block is zero, however full
    the diagonal blocks are."""
    nn, h = 16, 8
    A = _pivot_block(nn, 95 + p, rows=50)
    sg = W.signs_block(nn, p)
    Ao, Wp, nrot, passes, st = orc.inner_solve(A, sg, _tol(nn), mode=1, order=order)
    assert st == 0 and passes == 1 and 0 < nrot <= h * h
    _congruence_checks(A, sg, Ao, Wp)
    Z = A.copy()
    Z[:h, h:] = 0.0
    Z[h:, :h] = 0.0
    Zo, Wz, nz, _, st = orc.inner_solve(Z, sg, _tol(nn), mode=1, order=order)
    assert st == 0 and nz == 0 and np.array_equal(Wz, np.eye(nn)) and np.array_equal(Zo, Z)


@pytest.mark.parametrize("order", ORDERS)
@pytest.mark.parametrize("mode", [1, 2])
def test_inner_solve_visits_every_cross_pair_once(orc, order, mode):
    """A pass visits every pair of the off-diagonal block once (Sec. 5): a
    diagonal block with one coupling at (k, h + j), anywhere in that block,
    is rotated exactly once, and the coupling ends exactly zero."""
    nn, h = 16, 8
    D = np.diag(np.arange(1.0, nn + 1.0))
    sg = W.signs_block(nn, 5)
    for k in range(h):
        for j in range(h):
            A = D.copy()
            A[k, h + j] = A[h + j, k] = 0.25
            Ao, Wp, nrot, passes, st = orc.inner_solve(A, sg, _tol(nn), mode=mode, order=order)
            assert st == 0 and nrot == 1 and Ao[k, h + j] == 0.0, (k, j, nrot)


@pytest.mark.parametrize("order", ORDERS)
@pytest.mark.parametrize("mode", [1, 2])
def test_inner_solve_one_pass_invariants(orc, order, mode):
    """One pass (the cross pass, or one pass over the whole strict upper
    triangle, Sec. 5): the congruence checks on graded blocks with mixed
    signs; with J = I every rotation is orthogonal, so the Frobenius norm of
    the block is kept and the off-diagonal mass can only fall (each rotation
    removes 2 a_pq^2 of it); the pair the order visits last is exactly zero."""
    for nn, seed in ((8, 1), (32, 2), (64, 3)):
        h = nn // 2
        A = _pivot_block(nn, 300 + seed, lo=-3)
        for sg in (W.signs_block(nn, h), W.signs_random(np.random.default_rng(seed), nn, nn // 3),
                   np.ones(nn, dtype=np.int8)):
            Ao, Wp, nrot, passes, st = orc.inner_solve(A, sg, _tol(nn), mode=mode, order=order)
            assert st == 0 and nrot > 0
            _congruence_checks(A, sg, Ao, Wp)
            if np.all(sg == 1):
                assert abs(np.linalg.norm(Ao) - np.linalg.norm(A)) <= 4 * nn * U * np.linalg.norm(A)
                off = lambda X: np.linalg.norm(X - np.diag(np.diag(X)))  # noqa: E731
                assert off(Ao) <= off(A)
            if order == "cyclic":
                p, q = (h - 1, nn - 1) if mode == 1 else (nn - 2, nn - 1)
                assert Ao[p, q] == 0.0 or abs(Ao[p, q]) < _tol(nn) * np.sqrt(Ao[p, p] * Ao[q, q])


# --------------------------------------------------------------------------
# Pin 9: orderings and the blocked method agree (noise floor of the method)
# --------------------------------------------------------------------------
def test_orderings_and_blocked_agree(orc):
    G, J = W.graded(128, decades=6, seed=2)
    n = 128
    ref = orc.hsvd(G, J, _tol(n), 40)
    assert ref["status"] == 0
    runs = [orc.hsvd(G, J, _tol(n), 40, order="modulus", sort=True),
            orc.block_hsvd(G, J, 8, _tol(n), 40, inner_mode=1),
            orc.block_hsvd(G, J, 16, _tol(n), 40, inner_mode=0, inner_max_passes=10)]
    for r in runs:
        assert r["status"] == 0
        for s in (1, -1):
            a = np.sort(r["sigma"][J == s])
            b = np.sort(ref["sigma"][J == s])
            assert np.max(np.abs(a - b) / b) <= 1e-12
        orth, junit, resid = _invariants(G, J, r)
        assert orth <= 1e-12 * n and junit <= 1e-12 * n and resid <= 1e-12 * n


# --------------------------------------------------------------------------
# Statuses (error behaviour of the oracle)
# --------------------------------------------------------------------------
def test_statuses(orc):
    G, J = W.gaussian(16, seed=5)
    bad = G.copy()
    bad[3, 4] = np.nan
    assert orc.hsvd(bad, J, _tol(16), 10)["status"] == orc.ORC_NONFINITE
    assert orc.hsvd(G[:10, :], J, _tol(16), 10)["status"] == orc.ORC_ARG
    assert orc.hsvd(G, J, _tol(16), 1)["status"] == orc.ORC_NOT_CONVERGED
    # two equal columns of opposite sign: the pair has |zeta| = 1, there is no
    # hyperbolic rotation (M = G J G^T loses rank, Sec. 1)
    Gr = np.asfortranarray(np.repeat(G[:, :1], 2, axis=1))
    assert orc.hsvd(Gr, np.array([1, -1]), _tol(2), 30)["status"] == orc.ORC_RANK
    Gz = G.copy()
    Gz[:, 7] = 0.0
    assert orc.hsvd(Gz, J, _tol(16), 30)["status"] == orc.ORC_RANK


def test_modulus_parallel_mode_equals_serial():
    """The OpenMP modulus-parallel mode spreads the disjoint pairs of a step
    over threads: the result is the serial modulus order's, bit for bit."""
    import oracle

    oracle.build()
    G, J = W.gaussian(96, m=110, p=40, seed=17)
    tol = 96 * U
    oracle.set_threads(1)
    r1 = oracle.hsvd(G, J, tol, 30, order="modulus", sort=True)
    oracle.set_threads(4)
    r4 = oracle.hsvd(G, J, tol, 30, order="modulus", sort=True)
    oracle.set_threads(0)
    assert r1["status"] == 0 and r1["sweeps"] == r4["sweeps"]
    assert np.array_equal(r1["sigma"], r4["sigma"]) and np.array_equal(r1["V"], r4["V"])
