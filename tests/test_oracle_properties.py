"""Property-based checks of the oracle on random small inputs (hypothesis
draws shapes, signatures, scalings and seeds): every solver form returns the
HSVD invariants and LAPACK's eigenvalues of G J G^T, and with J = I LAPACK's
singular values; the symmetric factorisation reproduces M and its inertia;
the hyperbolic QR satisfies its defining identities; the split-precision
Gram model stays within its error bound.  CPU only; skipped where
hypothesis is not installed."""
import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings  # noqa: E402
from hypothesis import strategies as st  # noqa: E402

U = 2.0 ** -53


@st.composite
def factors(draw):
    n = draw(st.integers(1, 12))
    m = draw(st.integers(n, n + 6))
    seed = draw(st.integers(0, 2 ** 31 - 1))
    decades = draw(st.sampled_from([0.0, 2.0, 5.0]))
    rng = np.random.default_rng(seed)
    G = rng.standard_normal((m, n)) * 10.0 ** (-decades * rng.random(n))[None, :]
    J = np.where(rng.random(n) < draw(st.sampled_from([0.0, 0.5, 1.0])), 1, -1).astype(np.int8)
    return np.asfortranarray(G), J


def _check(G, J, r):
    m, n = G.shape
    assert r["status"] == 0
    s, Uo, V = r["sigma"], r["U"], r["V"]
    Jd = J.astype(np.float64)
    nv = max(1.0, float(np.max(np.abs(V))))
    assert np.max(np.abs(G @ V - Uo * s[None, :])) <= 64 * m * U * np.linalg.norm(G) * nv
    assert np.max(np.abs(Uo.T @ Uo - np.eye(n))) <= 64 * n * U
    assert np.max(np.abs(V.T @ (Jd[:, None] * V) - np.diag(Jd))) <= 64 * n * U * nv ** 2
    ev = np.sort(np.linalg.eigvalsh((G * Jd[None, :]) @ G.T))
    lam = np.sort(np.concatenate([s ** 2 * Jd, np.zeros(m - n)]))
    assert np.max(np.abs(lam - ev)) <= 64 * m * U * np.linalg.norm(G) ** 2


@settings(max_examples=60, deadline=None)
@given(factors(), st.sampled_from(["cyclic", "modulus", "modulus-sorted", "block1", "block2"]))
def test_every_form_returns_the_hsvd(orc, fj, form):
    G, J = fj
    n = G.shape[1]
    tol = max(n, 2) * U
    if form.startswith("block"):
        b = int(form[5:])
        r = orc.block_hsvd(G, J, b, tol, 60, inner_mode=1, sort=False)
    else:
        r = orc.hsvd(G, J, tol, 60, order=form.split("-")[0], sort=form.endswith("sorted"))
    _check(G, J, r)


@settings(max_examples=40, deadline=None)
@given(factors())
def test_identity_signature_gives_lapack_singular_values(orc, fj):
    G, _ = fj
    n = G.shape[1]
    r = orc.hsvd(G, np.ones(n, dtype=np.int8), max(n, 2) * U, 60)
    assert r["status"] == 0
    sv = np.linalg.svd(G, compute_uv=False)
    # LAPACK's SVD is accurate relative to sigma_max (a graded factor's small
    # values carry its normwise error), so compare on that scale
    assert np.max(np.abs(np.sort(r["sigma"])[::-1] - sv)) <= 64 * G.shape[0] * U * sv[0]


@st.composite
def symmetric(draw):
    n = draw(st.integers(1, 10))
    seed = draw(st.integers(0, 2 ** 31 - 1))
    kind = draw(st.sampled_from(["random", "saddle", "graded"]))
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n))
    M = (A + A.T) / 2
    if kind == "saddle" and n % 2 == 0:
        M[: n // 2, : n // 2] = 0.0
        M[n // 2:, n // 2:] = 0.0
    if kind == "graded":
        d = 10.0 ** (-3 * rng.random(n))
        M = M * d[:, None] * d[None, :]
    return np.asfortranarray(M)


@settings(max_examples=60, deadline=None)
@given(symmetric())
def test_symmetric_factorisation_properties(orc, M):
    """M = G J G^T to rounding, and the signs of J are the inertia of M."""
    n = M.shape[0]
    ev = np.linalg.eigvalsh(M)
    hypothesis.assume(np.min(np.abs(ev)) > 1e-8 * np.max(np.abs(ev)))  # numerically nonsingular
    G, J, perm, st_ = orc.sym_factor(M)
    assert st_ == 0
    R = (G * J.astype(np.float64)[None, :]) @ G.T - M
    assert np.max(np.abs(R)) <= 100 * n * U * np.max(np.abs(G)) ** 2
    assert int((J > 0).sum()) == int((ev > 0).sum())
    assert sorted(perm.tolist()) == list(range(n))


@settings(max_examples=60, deadline=None)
@given(st.integers(1, 8), st.integers(0, 6), st.integers(0, 2 ** 31 - 1))
def test_hyperbolic_qr_properties(orc, m, extra, seed):
    """T A C = [R; 0] and T^T Jh T = J, with T formed explicitly, R block
    upper triangular, Jh a permutation of J, whenever the factorisation
    exists."""
    n = m + extra
    rng = np.random.default_rng(seed)
    A = np.asfortranarray(rng.standard_normal((n, m)))
    J = np.where(rng.random(n) < 0.5, 1, -1).astype(np.int8)
    q = orc.hyp_qr(A, J)
    assert q["status"] in (0, orc.ORC_RANK)
    hypothesis.assume(q["status"] == 0)
    T = orc.hyp_qr_apply_tt(q, np.eye(n)).T
    R, Jh = q["R"], q["Jh"].astype(np.float64)
    nt = max(1.0, float(np.max(np.abs(T))))
    assert np.max(np.abs(T @ A[:, q["cperm"]] - np.vstack([R, np.zeros((n - m, m))]))) <= 64 * n * U * nt * np.max(
        np.abs(A))
    assert np.max(np.abs(T.T @ (Jh[:, None] * T) - np.diag(J.astype(np.float64)))) <= 64 * n * U * nt ** 2
    bs = q["bsize"]
    for j in range(m):  # block upper triangular: 1 x 1 pivots and 2 x 2 blocks (2, 0)
        assert np.all(R[j + (2 if bs[j] == 2 else 1):, j] == 0.0)
    assert sorted(q["Jh"].tolist()) == sorted(J.tolist())


@settings(max_examples=40, deadline=None)
@given(st.integers(1, 600), st.integers(0, 2 ** 31 - 1), st.sampled_from([0.0, 3.0, 8.0]))
def test_split_gram_within_its_bound(rows, seed, spread):
    """The split-precision Gram model on random windows: symmetric, and each
    entry within 5.6 K 2^-55 2^(E_i + E_j) per window (plus the roundings) of
    the exact dot product."""
    from fractions import Fraction

    from oracle import split

    rng = np.random.default_rng(seed)
    P = rng.standard_normal((rows, 4)) * 10.0 ** rng.uniform(-spread, spread, size=(rows, 4))
    A = split.gram(P)
    assert np.array_equal(A, A.T)
    for i in range(4):
        for j in range(i, 4):
            exact = sum(Fraction(float(a)) * Fraction(float(b)) for a, b in zip(P[:, i], P[:, j]))
            bound = 2 * U * abs(A[i, j])
            for r0 in range(0, rows, split.WINDOW):
                w = P[r0:r0 + split.WINDOW]
                E = split.column_exponents(w)
                bound += 5.6 * w.shape[0] * 2.0 ** -55 * 2.0 ** int(E[i] + E[j]) + 2 * U * abs(float(w[:, i] @ w[:, j]))
            assert abs(Fraction(float(A[i, j])) - exact) <= Fraction(bound)
