"""The shortening front end (Sec. 1): G = Q R by the library's Householder
QR, the HSVD of R, U = Q [U_R; 0].  The QR is checked against LAPACK
(numpy), the shortened HSVD against the direct one and the oracle, and the
invariants are checked on the original G."""
import numpy as np
import pytest
import torch

import oracle
from paper_1008_1371_gb300 import workloads as W

pytestmark = pytest.mark.gpu
U64 = 2.0 ** -53


@pytest.fixture(scope="module")
def api():
    from paper_1008_1371_gb300 import api, build_lib

    build_lib.build()
    oracle.build()
    assert torch.cuda.is_available()
    return api


@pytest.mark.parametrize("m,n", [(700, 200), (257, 33), (64, 1), (96, 96), (1000, 320), (129, 64), (14000, 64), (40, 40)])
def test_qr_matches_lapack(api, m, n):
    """Panels on a 16-CTA cluster where their rows fit its shared memory
    (14000 rows do not: the one-CTA panel kernel takes them; 40 rows are
    too few for the cluster)."""
    rng = np.random.default_rng(m + n)
    G = np.asfortranarray(rng.standard_normal((m, n)) * 10.0 ** rng.uniform(-4, 2, n)[None, :])
    R, Q = api.hsvd_shorten_qr(torch.from_numpy(G).cuda())
    R, Q = R.cpu().numpy(), Q.cpu().numpy()
    Rn = np.linalg.qr(G, mode="r")  # LAPACK dgeqrf: the same sign convention for R_jj
    colnorm = np.linalg.norm(G, axis=0)
    assert np.allclose(np.tril(R, -1), 0.0, atol=0.0)
    assert np.max(np.abs(R - Rn) / colnorm[None, :]) <= 50 * m * U64
    assert np.max(np.abs(Q.T @ Q - np.eye(n))) <= 10 * m * U64
    assert np.max(np.linalg.norm(Q @ R - G, axis=0) / colnorm) <= 10 * m * U64


def _run(api, G, J, host=False, **kw):
    dev = torch.device("cpu") if host else torch.device("cuda:0")
    Gt = torch.from_numpy(np.asfortranarray(G)).to(dev)
    Jt = torch.from_numpy(J).to(dev)
    if host:
        Gt, Jt = Gt.pin_memory(), Jt.pin_memory()
    r = api.hsvd_solve_ex(Gt, Jt, api.make_opts(**kw))
    torch.cuda.synchronize()
    return r


def _err(J, a, b):
    e = 0.0
    for s in (1, -1):
        if np.any(J == s):
            x, y = np.sort(a[J == s]), np.sort(b[J == s])
            e = max(e, float(np.max(np.abs(x - y) / y)))
    return e


@pytest.mark.parametrize("m,n,method", [(600, 150, 1), (900, 300, 2), (2000, 512, 2), (333, 100, 0)])
def test_shortened_hsvd(api, m, n, method):
    G, J = W.graded(n, m=m, decades=3.0, seed=70 + n)
    a = _run(api, G, J, method=method, shorten=api.HSVD_SHORTEN_ALWAYS)
    d = _run(api, G, J, shorten=api.HSVD_SHORTEN_NEVER)  # the tall factor directly (blocked when it must)
    assert a.status == d.status == api.HSVD_OK and a.shortened == 1 and d.shortened == 0
    s = a.sigma.cpu().numpy()
    assert _err(J, s, d.sigma.cpu().numpy()) <= 1e-12
    ref = oracle.hsvd(G, J, n * U64, 40, order="modulus", sort=True, want_u=False, want_v=False)
    assert ref["status"] == 0 and _err(J, s, ref["sigma"]) <= 1e-12
    U, V = a.U.cpu().numpy(), a.V.cpu().numpy()
    Jd = np.diag(J.astype(float))
    assert np.max(np.abs(U.T @ U - np.eye(n))) <= 1e-12 * n
    assert np.max(np.abs(V.T @ Jd @ V - Jd)) / max(1.0, np.max(np.abs(V)) ** 2) <= 1e-12 * n
    res = np.linalg.norm(G @ V - U * s[None, :], axis=0) / (np.linalg.norm(G) * np.linalg.norm(V, axis=0))
    assert np.max(res) <= 1e-12 * n


def test_shortening_choice_and_host_arrays(api):
    """Automatic shortening when 4m >= 5n; host arrays take the same path."""
    G, J = W.gaussian(200, m=260, seed=71)   # 4m = 1040 >= 1000
    r = _run(api, G, J)
    assert r.status == api.HSVD_OK and r.shortened == 1
    G2, J2 = W.gaussian(200, m=240, seed=72)  # 4m = 960 < 1000
    r2 = _run(api, G2, J2)
    assert r2.status == api.HSVD_OK and r2.shortened == 0
    h = _run(api, G, J, host=True)
    assert h.shortened == 1 and torch.equal(h.sigma, r.sigma.cpu()) and torch.equal(h.U, r.U.cpu())
    # a square factor is never shortened
    G3, J3 = W.gaussian(128, seed=73)
    assert _run(api, G3, J3, shorten=api.HSVD_SHORTEN_ALWAYS).shortened == 0
