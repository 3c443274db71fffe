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


@pytest.mark.parametrize("n", [8, 31])
def test_singular_matrix(api, n):
    """The zero matrix, and a saddle point matrix of odd order (rank n - 1)."""
    M = np.zeros((n, n)) if n == 8 else _sym("saddle", n, 38)
    with pytest.raises(api.HsvdError) as e:
        api.hsvd_sym_factor(torch.from_numpy(np.asfortranarray(M)).cuda())
    assert e.value.status == api.HSVD_ERR_RANK
