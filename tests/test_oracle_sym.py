"""Pins for the oracle's symmetric indefinite factorisation M = G J G^T
(Bunch-Parlett pivoting): the residual against M, Sylvester's law of inertia
against LAPACK's eigenvalues, the pivot rule on small matrices worked by
hand, and planted mistakes that the residual catches.  No GPU needed."""
import os

import numpy as np
import pytest

U = 2.0 ** -53
SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "hsvd_oracle.c")


def _sym(kind, n, seed):
    rng = np.random.default_rng(seed)
    if kind == "random":
        A = rng.standard_normal((n, n))
        return (A + A.T) / 2
    if kind == "saddle":
        h = n // 2
        B = rng.standard_normal((h, n - h))
        M = np.zeros((n, n))
        M[:h, h:] = B
        M[h:, :h] = B.T
        return M
    A = rng.standard_normal((n, n))
    return A @ A.T + n * np.eye(n)


def _residual(G, J, M):
    return np.max(np.abs((G * J[None, :].astype(float)) @ G.T - M)) / np.max(np.abs(M))


@pytest.mark.parametrize("kind,n", [("random", 1), ("random", 2), ("random", 7), ("random", 60), ("saddle", 40),
                                    ("saddle", 10), ("definite", 30)])
def test_residual_and_inertia(orc, kind, n):
    M = _sym(kind, n, 20 + n)
    G, J, perm, st = orc.sym_factor(M)
    assert st == 0
    assert _residual(G, J, M) <= 50 * n * U
    ev = np.linalg.eigvalsh(M)
    assert int((J > 0).sum()) == int((ev > 0).sum())  # Sylvester's law of inertia
    assert sorted(perm.tolist()) == list(range(n))
    if kind == "definite":
        assert np.all(J == 1)


def test_pivot_rule_by_hand(orc):
    """[[0, 2], [2, 0]]: no diagonal to pivot on, a 2 x 2 pivot; its block has
    eigenvalues +2 and -2, so J = (+1, -1) and G G^T's scale is 2.
    [[4, 1], [1, 0.1]]: |a_00| = 4 >= alpha 4, a 1 x 1 pivot on index 0 with
    L = [1; 1/4], D = diag(4, 0.1 - 1/4): J = (+1, -1) and G = [[2, 0], [0.5, sqrt(0.15)]]."""
    G, J, perm, st = orc.sym_factor(np.array([[0.0, 2.0], [2.0, 0.0]]))
    assert st == 0 and sorted(J.tolist()) == [-1, 1]
    assert _residual(G, J, np.array([[0.0, 2.0], [2.0, 0.0]])) <= 4 * U
    G, J, perm, st = orc.sym_factor(np.array([[4.0, 1.0], [1.0, 0.1]]))
    assert st == 0 and J.tolist() == [1, -1] and perm.tolist() == [0, 1]
    assert np.allclose(G, [[2.0, 0.0], [0.5, np.sqrt(0.15)]], rtol=0, atol=4 * U)
    # the larger diagonal entry is brought to the front
    G, J, perm, st = orc.sym_factor(np.array([[0.1, 1.0], [1.0, 4.0]]))
    assert st == 0 and perm.tolist() == [1, 0]


def _numerical_rank(M):
    ev = np.linalg.eigvalsh(M)
    return int(np.sum(np.abs(ev) > M.shape[0] * U * max(np.max(np.abs(ev)), 1e-300))), ev


@pytest.mark.parametrize("case", ["zero", "diag", "saddle9", "saddle31", "block", "pow2"])
def test_singular_postprocessing(orc, case):
    """A singular M (Sec. 1, the factorisation with postprocessing; reading
    R16): the factorisation stops once the trailing matrix is zero, with rank
    r = the number of nonzero eigenvalues (LAPACK), M = G_r J_r G_r^T for the
    first r columns, G_r of full column rank, J_r's inertia that of M, and
    zeros past r."""
    rng = np.random.default_rng(77)
    if case == "zero":
        M = np.zeros((5, 5))
    elif case == "diag":
        M = np.diag([1.0, -1.0, 0.0])
    elif case.startswith("saddle"):  # odd order: rank n - 1
        M = _sym("saddle", int(case[6:]), 38)
    elif case == "block":  # [[A, 0], [0, 0]] with A random symmetric of order 7
        M = np.zeros((12, 12))
        A = rng.standard_normal((7, 7))
        M[:7, :7] = A + A.T
        p = rng.permutation(12)
        M = M[np.ix_(p, p)]
    else:  # v v^T - w w^T with power-of-two entries: every step exact
        v = np.array([1.0, 2.0, 0.0, 4.0, 0.5, 0.0])
        w = np.array([0.0, 1.0, 8.0, 0.0, 2.0, 0.25])
        M = np.outer(v, v) - np.outer(w, w)
    n = M.shape[0]
    G, J, perm, st, r = orc.sym_factor(M, want_rank=True)
    want, ev = _numerical_rank(M)
    assert st == 0 and r == want, (r, want)
    assert np.all(G[:, r:] == 0.0) and np.all(J[r:] == 0) and set(J[:r].tolist()) <= {-1, 1}
    Gr, Jr = G[:, :r], J[:r].astype(float)
    assert np.max(np.abs((Gr * Jr[None, :]) @ Gr.T - M)) <= 50 * n * U * max(np.max(np.abs(M)), 1.0)
    assert int((Jr > 0).sum()) == int((ev > n * U * np.max(np.abs(ev) + 1e-300)).sum())
    if r:
        assert np.linalg.svd(Gr, compute_uv=False)[-1] > 1e-8 * np.linalg.norm(Gr)


def test_non_finite_is_rank_error(orc):
    M = np.eye(4)
    M[2, 1] = M[1, 2] = np.nan
    assert orc.sym_factor(M)[3] == orc.ORC_RANK


MUTANTS = {
    "alpha_test_inverted": ("if (k == n - 1 || omax <= 0.0 || dmax >= alpha * mu0) {",
                            "if (k == n - 1 || omax <= 0.0 || dmax < alpha * mu0) {"),
    "inverse_offdiag_sign": ("            i01 = -d01 / det;\n            i11 = d00 / det;\n        }\n        /* trailing",
                             "            i01 = d01 / det;\n            i11 = d00 / det;\n        }\n        /* trailing"),
    "column_swap_dropped": ("    for (int i = k; i < n; ++i) { /* columns a, b in the trailing rows but a and b */",
                            "    for (int i = n; i < n; ++i) { /* columns a, b in the trailing rows but a and b */"),
    "schur_angle_sign": ("                    c1 = -sn * sqrt(fabs(l1));", "                    c1 = sn * sqrt(fabs(l1));"),
    "rank_stop_dropped": ("        if (mu0 == 0.0) break; /* R16: the trailing matrix is zero, M has rank k */\n", ""),
}


def _battery_fails(orc, lib):
    for kind, n in (("random", 30), ("saddle", 20), ("random", 9), ("saddle", 9)):
        M = _sym(kind, n, 5 + n)
        G, J, perm, st = orc.sym_factor(M, lib=lib)
        ev = np.linalg.eigvalsh(M)
        pos = int((ev > n * U * np.max(np.abs(ev))).sum())
        if st != 0 or not np.all(np.isfinite(G)) or _residual(G, J, M) > 50 * n * U \
                or int((J > 0).sum()) != pos:
            return True
    return False


def test_battery_passes_on_oracle(orc):
    assert not _battery_fails(orc, orc.load())


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_residual_catches_planted_mistake(orc, tmp_path, name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, name
    path = tmp_path / ("orc_%s.c" % name)
    path.write_text(src.replace(old, new))
    lib = orc.load(orc.build(force=True, src=str(path), out=str(tmp_path / ("liborc_%s.so" % name))))
    assert _battery_fails(orc, lib), "planted mistake %s went unnoticed" % name
