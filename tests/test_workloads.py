"""The seeded input generators: the shapes, signatures and structure each one
promises, checked with LAPACK (the generators feed both the CUDA path and the
oracle, so a wrong input would fool both alike).  CPU only."""
import numpy as np
import pytest

from paper_1008_1371_gb300 import workloads as W


def _signed(J):
    return np.asarray(J).astype(np.float64)


def test_seeded_and_column_major():
    for gen in (lambda s: W.gaussian(24, m=30, p=7, seed=s), lambda s: W.graded(24, seed=s),
                lambda s: W.haar(24, seed=s), lambda s: W.paper(24, seed=s)[:2], lambda s: W.wide(8, 20, seed=s)[:2]):
        G1, J1 = gen(3)
        G2, J2 = gen(3)
        G3, _ = gen(4)
        assert np.array_equal(G1, G2) and np.array_equal(J1, J2) and not np.array_equal(G1, G3)
        assert G1.flags.f_contiguous and G1.dtype == np.float64 and J1.dtype == np.int8
        assert set(np.unique(J1)) <= {-1, 1} and J1.shape == (G1.shape[1],)


def test_signature_counts():
    G, J = W.gaussian(40, p=13, seed=1)
    assert int((J > 0).sum()) == 13 and np.all(J[:13] == 1)
    _, J = W.haar(64, p=20, seed=2)
    assert int((J > 0).sum()) == 20
    for n, p in ((16, 0), (17, 17), (30, 11)):
        _, J, _ = W.paper(n, p=p, seed=5)
        assert int((J > 0).sum()) == p


def test_graded_columns():
    """G = B diag(10^(-d i/n)): column norms fall by d decades across G, and
    the powers of ten are the correctly rounded ones."""
    n, d = 64, 6.0
    G, _ = W.graded(n, decades=d, seed=2)
    assert G.shape == (n, n)
    s = np.array([10.0 ** (-d * i / n) for i in range(n)])
    ratio = np.linalg.norm(G, axis=0) / s
    assert np.max(ratio) / np.min(ratio) < 10.0  # N(0,1) column norms, about sqrt(n) each
    from decimal import Context, Decimal
    ctx = Context(prec=40)
    for x in (-6.0 * 5 / 64, -3.0, -0.1):
        assert W._pow10([x])[0] == float(ctx.power(Decimal(10), Decimal(repr(x))))


@pytest.mark.parametrize("n,p", [(32, 16), (48, 0), (40, 40), (64, 9)])
def test_paper_known_spectrum(n, p):
    """sigma = sqrt|lambda| by construction: the eigenvalues of G J G^T
    (LAPACK) are sigma^2 J, and the spectrum has Table 5.2's range."""
    G, J, sig = W.paper(n, p=p, seed=n + p)
    ev = np.sort(np.linalg.eigvalsh((G * _signed(J)[None, :]) @ G.T))
    lam = np.sort(sig ** 2 * _signed(J))
    assert np.max(np.abs(ev - lam) / np.abs(lam)) <= 1e-10
    a = W.paper_a(n)
    assert np.all(sig ** 2 <= a) and np.all(sig ** 2 >= a * 1e-5)


@pytest.mark.parametrize("m,n,p", [(8, 20, 10), (16, 64, 60), (12, 12, 3), (1, 5, 2)])
def test_wide_known_spectrum(m, n, p):
    G, J, lam = W.wide(m, n, p, seed=m * n)
    assert G.shape == (m, n) and int((J > 0).sum()) == p
    ev = np.sort(np.linalg.eigvalsh((G * _signed(J)[None, :]) @ G.T))
    assert np.max(np.abs(ev - lam) / np.abs(lam)) <= 1e-10


def test_haar_singular_values():
    """G = Q1 diag(sigma) Q2: LAPACK's singular values are log-uniform in
    [lo, hi]."""
    G, _ = W.haar(48, lo=1e-4, hi=1.0, seed=3)
    sv = np.linalg.svd(G, compute_uv=False)
    assert sv.max() <= 1.0 + 1e-12 and sv.min() >= 1e-4 * (1 - 1e-9)


def test_batch_shapes():
    facs = W.batch(50, nmin=16, nmax=40, seed=4)
    assert len(facs) == 50
    for G, J in facs:
        m, n = G.shape
        assert m == n and 16 <= n <= 40 and J.shape == (n,)
