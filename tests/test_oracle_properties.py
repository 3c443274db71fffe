"""Property-based checks of the oracle on random small factors (hypothesis
draws shapes, signatures, scalings and seeds): every solver form returns the
HSVD invariants and LAPACK's eigenvalues of G J G^T, and with J = I LAPACK's
singular values.  CPU only; skipped where hypothesis is not installed."""
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
