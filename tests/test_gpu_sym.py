"""The symmetric indefinite factorisation M = G J G^T (Bunch-Parlett pivoting)
and the eigensolver built on it (factorisation, then the HSVD of G), checked
against what holds independently: the residual of G J G^T, Sylvester's law of
inertia (the signs of J count M's positive eigenvalues), and LAPACK's
eigenvalues and eigenvector residuals."""
import numpy as np
import pytest
import torch

from paper_1008_1371_gb300 import workloads as W

pytestmark = pytest.mark.gpu
U64 = 2.0 ** -53


@pytest.fixture(scope="module")
def api():
    from paper_1008_1371_gb300 import api, build_lib

    build_lib.build()
    assert torch.cuda.is_available()
    return api


def _sym(kind, n, seed):
    rng = np.random.default_rng(seed)
    if kind == "random":
        A = rng.standard_normal((n, n))
        return (A + A.T) / 2
    if kind == "saddle":  # zero diagonal blocks (n even, so M is nonsingular): 2 x 2 pivots are forced
        h = n // 2
        B = rng.standard_normal((h, n - h))
        M = np.zeros((n, n))
        M[:h, h:] = B
        M[h:, :h] = B.T
        return M
    if kind == "definite":
        A = rng.standard_normal((n, n))
        return A @ A.T + n * np.eye(n)
    if kind == "paper":  # the paper's test spectrum: M = G J G^T, lambda = sigma^2 J
        G, J, _ = W.paper(n, seed=seed)
        return (G * J[None, :].astype(float)) @ G.T
    raise ValueError(kind)


@pytest.mark.parametrize("kind,n", [("random", 5), ("random", 33), ("random", 100), ("random", 257),
                                    ("saddle", 64), ("saddle", 30), ("definite", 80), ("paper", 160), ("random", 1)])
def test_factor_residual_and_inertia(api, kind, n):
    M = _sym(kind, n, 7 + n)
    G, J = api.hsvd_sym_factor(torch.from_numpy(np.asfortranarray(M)).cuda())
    G, J = G.cpu().numpy(), J.cpu().numpy().astype(float)
    R = (G * J[None, :]) @ G.T - M
    assert np.max(np.abs(R)) <= 50 * n * U64 * max(np.max(np.abs(M)), 1e-300)
    ev = np.linalg.eigvalsh(M)
    assert int((J > 0).sum()) == int((ev > 0).sum())  # Sylvester's law of inertia
    if kind == "definite":
        assert np.all(J > 0)


@pytest.mark.parametrize("kind,n", [("random", 33), ("saddle", 64), ("random", 100), ("definite", 50)])
def test_factor_matches_oracle(api, kind, n):
    """The same pivots and the same arithmetic as the CPU oracle's Bunch-Parlett
    factorisation: J equal, G equal bit for bit."""
    import oracle

    M = _sym(kind, n, 3 + n)
    G, J = api.hsvd_sym_factor(torch.from_numpy(np.asfortranarray(M)).cuda())
    Go, Jo, perm, st = oracle.sym_factor(M)
    assert st == 0
    assert np.array_equal(J.cpu().numpy(), Jo)
    assert np.array_equal(G.cpu().numpy(), Go)


@pytest.mark.parametrize("kind,n", [("random", 96), ("saddle", 128), ("paper", 288), ("random", 513)])
def test_eig_against_lapack(api, kind, n):
    M = _sym(kind, n, 11 + n)
    lam, U, info = api.hsvd_sym_eig(torch.from_numpy(np.asfortranarray(M)).cuda())
    assert info.status == api.HSVD_OK
    lam, U = lam.cpu().numpy(), U.cpu().numpy()
    ev = np.linalg.eigvalsh(M)
    nrm = np.max(np.abs(ev))
    assert np.max(np.abs(np.sort(lam) - ev)) <= 10 * n * U64 * nrm
    assert np.max(np.abs(U.T @ U - np.eye(n))) <= 1e-12 * n
    assert np.max(np.linalg.norm(M @ U - U * lam[None, :], axis=0)) <= 10 * n * U64 * nrm
    if kind == "paper":  # the known spectrum, value by value
        Gp, Jp, sig = W.paper(n, seed=11 + n)
        ref = np.sort(sig ** 2 * Jp)
        assert np.max(np.abs(np.sort(lam) - ref) / np.abs(ref)) <= 1e-10


def _singular(case):
    rng = np.random.default_rng(91)
    if case == "zero":
        return np.zeros((8, 8))
    if case == "saddle31":  # odd order: rank 30
        return _sym("saddle", 31, 38)
    if case == "block":  # [[A, 0], [0, 0]], A random symmetric of order 40, permuted
        M = np.zeros((64, 64))
        A = rng.standard_normal((40, 40))
        M[:40, :40] = A + A.T
        p = rng.permutation(64)
        return M[np.ix_(p, p)]
    v = np.array([1.0, 2.0, 0.0, 4.0, 0.5, 0.0])  # v v^T - w w^T, every step exact
    w = np.array([0.0, 1.0, 8.0, 0.0, 2.0, 0.25])
    return np.outer(v, v) - np.outer(w, w)


@pytest.mark.parametrize("case", ["zero", "saddle31", "block", "pow2"])
def test_singular_matrix_factor(api, case):
    """A singular M (the factorisation with postprocessing, Sec. 1): the GPU
    stops where the oracle stops, with the same rank, G and J bit for bit."""
    import oracle

    M = _singular(case)
    G, J, r = api.hsvd_sym_factor(torch.from_numpy(np.asfortranarray(M)).cuda(), want_rank=True)
    Go, Jo, perm, st, ro = oracle.sym_factor(M, want_rank=True)
    assert st == 0 and r == ro < M.shape[0]
    assert np.array_equal(J.cpu().numpy(), Jo) and np.array_equal(G.cpu().numpy(), Go)


@pytest.mark.parametrize("case", ["zero", "saddle31", "block", "pow2"])
def test_singular_matrix_eig(api, case):
    """The eigendecomposition of a singular M: r eigenvalues from the HSVD of
    the n x r factor, the others zero, with an orthonormal basis of the null
    space: against LAPACK, U^T U = I and M U = U diag(lambda)."""
    M = _singular(case)
    n = M.shape[0]
    lam, U, info = api.hsvd_sym_eig(torch.from_numpy(np.asfortranarray(M)).cuda())
    assert info.status == api.HSVD_OK
    lam, U = lam.cpu().numpy(), U.cpu().numpy()
    ev = np.linalg.eigvalsh(M)
    nrm = max(np.max(np.abs(ev)), 1.0)
    assert np.max(np.abs(np.sort(lam) - ev)) <= 10 * n * U64 * nrm
    assert np.max(np.abs(U.T @ U - np.eye(n))) <= 1e-12 * n
    assert np.max(np.linalg.norm(M @ U - U * lam[None, :], axis=0)) <= 10 * n * U64 * nrm


def test_non_finite_matrix(api):
    M = np.eye(6)
    M[2, 4] = M[4, 2] = np.inf
    with pytest.raises(api.HsvdError) as e:
        api.hsvd_sym_factor(torch.from_numpy(np.asfortranarray(M)).cuda())
    assert e.value.status == api.HSVD_ERR_RANK
