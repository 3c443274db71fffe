"""The wide case (m < n) on the GPU: the hyperbolic QR of G^T (Sec. 1)
shortens the factor to the square F = C R^T, whose HSVD gives sigma, U and
V = T^T [V_F; 0].  Checked against the CPU oracle's wide HSVD
(orc_wide_hsvd: the same reflectors and pivot rule, with the trailing J-Gram
recomputed at every step), against the known spectrum of the constructed
factors and LAPACK's eigenvalues of M = G J G^T, and by the invariants
G V = U Sigma, U^T U = I, V^T J V = diag(jout)."""
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


def _solve(api, G, J, **kw):
    dev = torch.device("cuda:0")
    r = api.hsvd_solve_ex(torch.from_numpy(np.asfortranarray(G)).to(dev), torch.from_numpy(J).to(dev),
                          api.make_opts(**kw), check=False)
    torch.cuda.synchronize()
    return r


def _lam(sigma, signs):
    return np.sort(sigma ** 2 * signs.astype(np.float64))


@pytest.mark.parametrize("m,n,p,seed", [(1, 3, 1, 1), (20, 37, 15, 2), (64, 100, 50, 3), (96, 256, 128, 4),
                                        (130, 300, 100, 5), (200, 201, 0, 6), (256, 512, 512, 7)])
def test_wide_matches_oracle_and_known_spectrum(api, m, n, p, seed):
    G, J, lam_true = W.wide(m, n, p=p, seed=seed)
    tol = m * U64
    r = _solve(api, G, J, tol=tol, max_sweeps=40)
    assert r.status == api.HSVD_OK and r.shortened == 2, api.hsvd_status_string(r.status)
    s, Uo, V, jo = r.sigma.cpu().numpy(), r.U.cpu().numpy(), r.V.cpu().numpy(), r.jout.cpu().numpy()
    assert s.shape == (m,) and Uo.shape == (m, m) and V.shape == (n, m) and set(np.unique(jo)) <= {-1, 1}
    ref = oracle.wide_hsvd(G, J, tol, 40)
    assert ref["status"] == 0
    # the same inertia and the same eigenvalues sigma^2 jout, per value
    assert np.sum(jo > 0) == np.sum(ref["Jout"] > 0) == np.sum(lam_true > 0)
    mine, theirs = _lam(s, jo), _lam(ref["sigma"], ref["Jout"])
    assert np.max(np.abs(mine - theirs) / np.abs(theirs)) <= 1e-11, np.max(np.abs(mine - theirs) / np.abs(theirs))
    assert np.max(np.abs(mine - lam_true) / np.abs(lam_true)) <= 1e-11
    # LAPACK's eigenvalues of M = G J G^T (absolute, M formed explicitly)
    ev = np.sort(np.linalg.eigvalsh((G * J[None, :].astype(float)) @ G.T))
    assert np.max(np.abs(ev - mine)) <= 16 * n * U64 * np.max(np.abs(ev))
    # invariants of Eq. 1.1 for the wide factor
    Jd = np.diag(J.astype(float))
    assert np.max(np.abs(Uo.T @ Uo - np.eye(m))) <= 1e-12 * m
    res = np.linalg.norm(G @ V - Uo * s[None, :], axis=0) / (np.linalg.norm(G) * np.linalg.norm(V, axis=0))
    assert np.max(res) <= 1e-12 * n
    jv = np.max(np.abs(V.T @ Jd @ V - np.diag(jo.astype(float)))) / max(1.0, np.max(np.abs(V)) ** 2)
    assert jv <= 1e-12 * n, jv


def test_wide_identity_signature_is_svd(api):
    """J = I: the hyperbolic QR is Householder QR with column pivoting and the
    result is the ordinary SVD of the wide G (LAPACK's singular values)."""
    G, _, _ = W.wide(80, 160, seed=11)
    J = np.ones(160, dtype=np.int8)
    r = _solve(api, G, J)
    assert r.status == 0 and np.all(r.jout.cpu().numpy() == 1)
    sv = np.linalg.svd(G, compute_uv=False)
    assert np.max(np.abs(np.sort(r.sigma.cpu().numpy())[::-1] - sv) / sv) <= 1e-12


def test_wide_forms_and_host_arrays(api):
    """The square F goes through the usual method choice: blocked FP64, the
    split-precision form and the pointwise method all give the same values;
    pinned host arrays give the device result bit for bit."""
    G, J, lam_true = W.wide(150, 300, p=120, seed=12)  # F = 150 x 150 fits one SM for the pointwise method
    base = _solve(api, G, J, method=api.HSVD_METHOD_BLOCKED, block_w=16)
    for kw in (dict(method=api.HSVD_METHOD_BLOCKED, precision=api.HSVD_PRECISION_BF16X8),
               dict(method=api.HSVD_METHOD_POINTWISE)):
        r = _solve(api, G, J, **kw)
        assert r.status == 0, kw
        assert np.max(np.abs(_lam(r.sigma.cpu().numpy(), r.jout.cpu().numpy()) - lam_true) / np.abs(lam_true)) <= 1e-11
    Gh = torch.from_numpy(np.asfortranarray(G)).pin_memory()
    Jh = torch.from_numpy(J).pin_memory()
    h = api.hsvd_solve_ex(Gh, Jh, api.make_opts(method=api.HSVD_METHOD_BLOCKED, block_w=16))
    assert h.status == 0 and h.sigma.device.type == "cpu"
    assert np.array_equal(h.sigma.numpy(), base.sigma.cpu().numpy())
    assert np.array_equal(h.V.numpy(), base.V.cpu().numpy()) and np.array_equal(h.jout.numpy(), base.jout.cpu().numpy())


def test_wide_singular_is_rank_error(api):
    """A zero row of G makes M = G J G^T singular: the hyperbolic QR meets a
    zero J-norm and the call returns HSVD_ERR_RANK, as the oracle does."""
    G, J, _ = W.wide(30, 70, seed=13)
    G = G.copy()
    G[7, :] = 0.0
    r = _solve(api, G, J)
    assert r.status == api.HSVD_ERR_RANK
    assert oracle.wide_hsvd(G, J, 30 * U64, 40)["status"] == oracle.ORC_RANK
