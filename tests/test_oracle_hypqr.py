"""Pins for the oracle's hyperbolic QR and the wide-factor HSVD built on it
(Sec. 1: a factor G whose transpose is tall is shortened by the hyperbolic
QR of G^T, the HSVD runs on the square R^T, and V is premultiplied by the
transformation).  The checks rest on facts fixed outside the oracle:

- with J = I the factorisation is Householder QR with column pivoting, so R
  and the pivot order must be LAPACK's (scipy's dgeqp3);
- 2 x 1 cases worked by hand (the row interchange, the sign of R);
- the defining identities T A C = [R; 0] and T^T Jh T = J, checked with T
  formed explicitly, and C^T A^T J A C = R^T Jh_1 R;
- Sylvester's law of inertia against LAPACK's eigenvalues of A^T J A;
- a wide factor with a known spectrum (workloads.wide) and LAPACK's
  eigenvalues of G J G^T, with the HSVD invariants G V = U Sigma,
  V^T J V = Jh_1, U^T U = I.

Planted mistakes in a copy of the C source are each caught.  No GPU needed."""
import os

import numpy as np
import pytest

from paper_1008_1371_gb300 import workloads as W

U = 2.0 ** -53
SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "hsvd_oracle.c")


def _signed(J):
    return np.asarray(J).astype(np.float64)


def _tall(n, m, p, seed):
    rng = np.random.default_rng(seed)
    A = np.asfortranarray(rng.standard_normal((n, m)) * np.exp2(rng.uniform(-3, 3, size=m))[None, :])
    return A, W.signs_random(rng, n, p)


def _explicit_t(orc, q, n, lib=None):
    """T itself: T^T = T^T I, column by column."""
    return orc.hyp_qr_apply_tt(q, np.eye(n), lib=lib).T


def _identity_errors(orc, A, J, lib=None):
    """Relative errors of T A C = [R; 0], T^T Jh T = J and
    C^T (A^T J A) C = R^T Jh_1 R, each scaled by the sizes of the terms."""
    n, m = A.shape
    q = orc.hyp_qr(A, J, lib=lib)
    assert q["status"] == 0
    R, Jh, C = q["R"], _signed(q["Jh"]), q["cperm"]
    T = _explicit_t(orc, q, n, lib=lib)
    AC = A[:, C]
    e1 = np.max(np.abs(T @ AC - np.vstack([R, np.zeros((n - m, m))]))) / (np.max(np.abs(T)) * np.max(np.abs(A)) * n)
    e2 = np.max(np.abs(T.T @ (Jh[:, None] * T) - np.diag(_signed(J)))) / (np.max(np.abs(T)) ** 2 * n)
    M = AC.T @ (_signed(J)[:, None] * AC)
    e3 = np.max(np.abs(M - R.T @ (Jh[:m, None] * R))) / (np.max(np.abs(A)) ** 2 * n)
    return q, e1, e2, e3


@pytest.mark.parametrize("seed", range(6))
def test_identity_signature_is_lapack_pivoted_qr(orc, seed):
    """J = I: no row interchange, and R and the column order are those of
    LAPACK's Householder QR with column pivoting (same sign convention,
    R_kk = -sign(x_k) ||x||)."""
    sl = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(400 + seed)
    n = int(rng.integers(8, 40))
    m = int(rng.integers(1, n + 1))
    A = rng.standard_normal((n, m)) * np.exp2(rng.uniform(-4, 4, size=m))[None, :]
    q = orc.hyp_qr(A, np.ones(n, dtype=np.int8))
    R, P = sl.qr(A, mode="r", pivoting=True)
    assert q["status"] == 0
    assert np.array_equal(q["cperm"], P) and np.array_equal(q["rswap"], np.arange(m))
    assert np.max(np.abs(q["R"] - R[:m, :m])) <= 8 * n * U * np.max(np.abs(R))
    assert np.all(q["Jh"] == 1)


def test_two_by_one_by_hand(orc):
    """A = [a; b], J = diag(1, -1), gamma = a^2 - b^2:
    [3; 1]: gamma = 8 > 0 = sign of row 0, no interchange, R = -sqrt(8);
    [1; 3]: gamma = -8, rows interchanged (Jh = (-1, 1)), x = [3; 1] and
    R = -sqrt(8); [-1; 3]: as before with x_k = 3 after the interchange;
    [2; -3] with J = diag(-1, 1): gamma = -4 + 9 = 5 > 0, interchange, then
    x = [-3; 2], R = +sqrt(5)."""
    J = np.array([1, -1], dtype=np.int8)
    for a, Jc, r, Jh, swap in (([3.0, 1.0], J, -np.sqrt(8.0), [1, -1], 0),
                               ([1.0, 3.0], J, -np.sqrt(8.0), [-1, 1], 1),
                               ([-1.0, 3.0], J, -np.sqrt(8.0), [-1, 1], 1),
                               ([2.0, -3.0], -J, np.sqrt(5.0), [1, -1], 1)):
        q = orc.hyp_qr(np.array(a).reshape(2, 1), Jc)
        assert q["status"] == 0
        assert abs(q["R"][0, 0] - r) <= 4 * U * abs(r), (a, q["R"])
        assert list(q["Jh"]) == Jh and q["rswap"][0] == swap
        T = _explicit_t(orc, q, 2)
        assert np.max(np.abs(T @ np.array(a) - [r, 0.0])) <= 32 * U * np.max(np.abs(T)) * 3
        assert np.max(np.abs(T.T @ np.diag(Jh) @ T - np.diag(Jc))) <= 32 * U * np.max(np.abs(T)) ** 2


def test_two_by_two_pivot_by_hand(orc):
    """A = [[1, 1], [1, -1]], J = diag(1, -1): both columns have J-norm^2 0
    and A^T J A = [[0, 2], [2, 0]] is nonsingular, so the only pivot is a
    2 x 2 block: R^T Jh_1 R = [[0, 2], [2, 0]] and Jh_1 has one sign of each
    kind (the eigenvalues are +-2)."""
    A = np.array([[1.0, 1.0], [1.0, -1.0]])
    J = np.array([1, -1], dtype=np.int8)
    q = orc.hyp_qr(A, J)
    assert q["status"] == 0 and list(q["bsize"]) == [2, 0]
    R, Jh = q["R"], _signed(q["Jh"])
    C = np.eye(2)[:, q["cperm"]]
    M = A.T @ np.diag(_signed(J)) @ A
    assert np.max(np.abs(R.T @ np.diag(Jh) @ R - C.T @ M @ C)) <= 16 * U
    assert sorted(q["Jh"].tolist()) == [-1, 1]
    r = orc.wide_hsvd(A.T, J, 4 * U, 20)
    assert r["status"] == 0
    assert np.allclose(np.sort(r["sigma"] ** 2 * r["Jout"]), [-2.0, 2.0], rtol=1e-15, atol=0)


def test_saddle_tall_factors_need_two_by_two_pivots(orc):
    """A = [B; B'] with J = diag(I, -I) and B' = B + a small perturbation:
    every column's J-norm^2 is small against the J-inner products, so 2 x 2
    pivots carry the factorisation, and the identities and the inertia
    hold."""
    rng = np.random.default_rng(5)
    B = rng.standard_normal((10, 6))
    A = np.asfortranarray(np.vstack([B, B + 0.3 * rng.standard_normal((10, 6))]))
    J = np.array([1] * 10 + [-1] * 10, dtype=np.int8)
    q, e1, e2, e3 = _identity_errors(orc, A, J)
    assert max(e1, e2, e3) <= 64 * U
    ev = np.linalg.eigvalsh(A.T @ (_signed(J)[:, None] * A))
    assert int(np.sum(q["Jh"][:6] > 0)) == int(np.sum(ev > 0))
    assert 2 in q["bsize"].tolist()


def test_breakdown_and_argument_errors(orc):
    """A zero trailing J-Gram (A^T J A singular, here 0) is ORC_RANK.  NaN, a
    bad sign, n < m are refused."""
    J = np.array([1, -1], dtype=np.int8)
    assert orc.hyp_qr(np.array([[1.0], [1.0]]), J)["status"] == orc.ORC_RANK
    assert orc.hyp_qr(np.array([[1.0], [np.nan]]), J)["status"] == orc.ORC_NONFINITE
    assert orc.hyp_qr(np.ones((2, 1)), np.array([1, 0], dtype=np.int8))["status"] == orc.ORC_ARG
    assert orc.wide_hsvd(np.ones((3, 2)), J, 1e-15)["status"] == orc.ORC_ARG


@pytest.mark.parametrize("n,m,p", [(12, 5, 6), (40, 17, 3), (40, 17, 37), (33, 33, 16), (64, 20, 0), (64, 1, 30)])
def test_defining_identities_and_inertia(orc, n, m, p):
    A, J = _tall(n, m, p, seed=n * 100 + m + p)
    q, e1, e2, e3 = _identity_errors(orc, A, J)
    assert e1 <= 16 * U and e2 <= 16 * U and e3 <= 16 * U, (e1, e2, e3)
    R, bs = q["R"], q["bsize"]
    # block upper triangular: 1 x 1 pivots, and 2 x 2 blocks marked (2, 0)
    for j in range(m):
        assert bs[j] in (1, 2, 0) and (bs[j] != 0 or (j > 0 and bs[j - 1] == 2))
        assert np.all(R[j + (2 if bs[j] == 2 else 1):, j] == 0.0)
    # Jh is J permuted; a first 1 x 1 pivot has the largest |J-norm^2| of A's columns
    assert sorted(q["Jh"].tolist()) == sorted(J.tolist())
    g = np.einsum("ij,i,ij->j", A, _signed(J), A)
    if bs[0] == 1:
        assert abs(R[0, 0] ** 2 - np.max(np.abs(g))) <= 8 * n * U * np.max(np.abs(A)) ** 2
    # Sylvester: the signs of R^T Jh_1 R are those of A^T J A's eigenvalues
    ev = np.linalg.eigvalsh(A.T @ (_signed(J)[:, None] * A))
    assert int(np.sum(q["Jh"][:m] > 0)) == int(np.sum(ev > 0))


@pytest.mark.parametrize("m,n,p", [(8, 20, 10), (20, 50, 25), (33, 40, 5), (16, 64, 60), (48, 48, 24), (1, 9, 4)])
@pytest.mark.parametrize("order", ["cyclic", "modulus"])
def test_wide_hsvd_known_spectrum(orc, m, n, p, order):
    """G = Q |Lambda|^(1/2) [I 0] K (K J-unitary): lambda = sigma^2 Jout
    matches the constructed spectrum to 1e-12, and the invariants hold."""
    G, J, lam = W.wide(m, n, p, seed=m + n + p)
    r = orc.wide_hsvd(G, J, max(m, 2) * U, 40, order=order)
    assert r["status"] == 0
    got = np.sort(r["sigma"] ** 2 * r["Jout"])
    assert np.max(np.abs(got - lam) / np.abs(lam)) <= 1e-12
    Uo, V, s = r["U"], r["V"], r["sigma"]
    nv = max(1.0, np.max(np.abs(V)))
    assert np.max(np.abs(G @ V - Uo * s)) <= 64 * n * U * np.max(np.abs(G)) * nv
    assert np.max(np.abs(V.T @ (_signed(J)[:, None] * V) - np.diag(_signed(r["Jout"])))) <= 64 * n * U * nv ** 2
    assert np.max(np.abs(Uo.T @ Uo - np.eye(m))) <= 64 * m * U


@pytest.mark.parametrize("seed", range(4))
def test_wide_hsvd_against_lapack_eigenvalues(orc, seed):
    """A random wide factor: lambda against LAPACK's eigenvalues of the
    formed G J G^T, to the accuracy of forming it (c u ||G||^2)."""
    rng = np.random.default_rng(900 + seed)
    m = int(rng.integers(2, 30))
    n = int(rng.integers(m, 60))
    G = np.asfortranarray(rng.standard_normal((m, n)))
    J = W.signs_random(rng, n, int(rng.integers(0, n + 1)))
    r = orc.wide_hsvd(G, J, m * U, 40)
    assert r["status"] == 0
    ev = np.sort(np.linalg.eigvalsh((G * _signed(J)[None, :]) @ G.T))
    got = np.sort(r["sigma"] ** 2 * r["Jout"])
    assert np.max(np.abs(got - ev)) <= 16 * n * U * np.max(np.abs(G)) ** 2 * n


def test_square_factor_agrees_with_direct_hsvd(orc):
    """m = n: the hyperbolic QR changes the factor, not the matrix G J G^T,
    so the eigenvalues equal those of the direct HSVD of G."""
    G, J, _ = W.paper(40, p=15, seed=12)
    r = orc.wide_hsvd(G, J, 40 * U, 40)
    d = orc.hsvd(G, J, 40 * U, 40)
    assert r["status"] == d["status"] == 0
    a = np.sort(r["sigma"] ** 2 * r["Jout"])
    b = np.sort(d["sigma"] ** 2 * _signed(J))
    assert np.max(np.abs(a - b) / np.abs(b)) <= 1e-12


# ---- planted mistakes --------------------------------------------------------

MUTANTS = {
    "beta_sign": ("const double beta = 2.0 / vsv;", "const double beta = -2.0 / vsv;"),
    "no_row_interchange": ("if (s[k] != sg) {", "if (0) {"),
    "alpha_sign": ("const double alpha = z[k] >= 0.0 ? -root : root;",
                   "const double alpha = z[k] >= 0.0 ? root : -root;"),
    "two_by_two_second_reflector_skips_x": ("status = hq_reduce(n, m, W, s, z, k + 1, k, v, &alpha2, &beta, &ip);",
                                            "status = hq_reduce(n, m, W, s, z, k + 1, k + 1, v, &alpha2, &beta, &ip);"),
    "update_plain_inner_product": ("for (int i = k; i < n; ++i) vsy += s[i] > 0 ? v[i] * y[i] : -(v[i] * y[i]);",
                                   "for (int i = k; i < n; ++i) vsy += v[i] * y[i];"),
    "apply_tt_drops_signature": ("for (int i = k; i < n; ++i) y[i] -= s[i] > 0 ? f * v[i] : -(f * v[i]);",
                                 "for (int i = k; i < n; ++i) y[i] -= f * v[i];"),
    "apply_tt_keeps_final_signature": ("            const int8_t t = s[k]; s[k] = s[ip]; s[ip] = t;\n        }\n    }\n"
                                       "    free(s);",
                                       "        }\n    }\n    free(s);"),
    "wide_rows_not_permuted": ("F[cperm[j] + (int64_t)l * m] = R[l + (int64_t)j * m];",
                               "F[j + (int64_t)l * m] = R[l + (int64_t)j * m];"),
}


def _battery(orc, lib):
    failed = []
    sl = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(3)
    A = rng.standard_normal((14, 6)) * np.exp2(rng.uniform(-3, 3, size=6))[None, :]
    q = orc.hyp_qr(A, np.ones(14, dtype=np.int8), lib=lib)
    R, P = sl.qr(A, mode="r", pivoting=True)
    if q["status"] != 0 or not np.array_equal(q["cperm"], P) or np.max(np.abs(q["R"] - R[:6, :6])) > 1e-13 * np.max(
            np.abs(R)):
        failed.append("lapack")
    q = orc.hyp_qr(np.array([[1.0], [3.0]]), np.array([1, -1], dtype=np.int8), lib=lib)
    if q["status"] != 0 or abs(q["R"][0, 0] + np.sqrt(8.0)) > 1e-15 or list(q["Jh"]) != [-1, 1]:
        failed.append("hand")
    for n, m, p in ((20, 8, 9), (30, 12, 25), (16, 8, 8)):
        A, J = _tall(n, m, p, seed=n + m)
        try:
            _, e1, e2, e3 = _identity_errors(orc, A, J, lib=lib)
            if max(e1, e2, e3) > 16 * U:
                failed.append("identities")
        except AssertionError:
            failed.append("identities-status")
    for m, n, p in ((10, 24, 12), (7, 30, 20)):
        G, J, lam = W.wide(m, n, p, seed=m * n)
        r = orc.wide_hsvd(G, J, m * U, 40, lib=lib)
        if r["status"] != 0:
            failed.append("wide-status")
            continue
        got = np.sort(r["sigma"] ** 2 * r["Jout"])
        nv = max(1.0, np.max(np.abs(r["V"])))
        if np.max(np.abs(got - lam) / np.abs(lam)) > 1e-12:
            failed.append("wide-spectrum")
        if np.max(np.abs(G @ r["V"] - r["U"] * r["sigma"])) > 64 * n * U * np.max(np.abs(G)) * nv:
            failed.append("wide-GV")
        if np.max(np.abs(r["V"].T @ (_signed(J)[:, None] * r["V"]) - np.diag(_signed(r["Jout"])))) > 64 * n * U * nv ** 2:
            failed.append("wide-VJV")
    return failed


def test_battery_passes_on_oracle(orc):
    assert _battery(orc, orc.load()) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_battery_catches_planted_mistake(orc, tmp_path, name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, name
    path = tmp_path / ("orc_%s.c" % name)
    path.write_text(src.replace(old, new))
    lib = orc.load(orc.build(force=True, src=str(path), out=str(tmp_path / ("liborc_%s.so" % name))))
    assert _battery(orc, lib), "planted mistake %s went unnoticed" % name
