"""The batched form (many factors, one persistent launch) against the CPU
oracle, and against the library's own single-factor pointwise solve.

Every factor is solved by the same per-factor code as the single pointwise
solve (pw_solve, Sec. 2 / Alg. 4.5, diagonal sorting of Sec. 4); the pairs of
a step are disjoint and each warp's reductions run over the same lanes, so
the results do not depend on the group width, the shared/global residency or
the queue position: they are compared bit for bit across those.  Against the
oracle (row-cyclic order, no sorting): sigma per sign group to the relative
tolerance 1e-12, and the invariants of Eq. 1.1."""
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


def _mixed(seed=11):
    """Factors of the sizes the batch meets: tiny, odd n (bordering), m > n,
    every residency class, all-plus and all-minus signatures."""
    rng = np.random.default_rng(seed)
    shapes = [(16, 16), (17, 17), (31, 24), (40, 40), (48, 33), (64, 64), (72, 71), (100, 100), (129, 128),
              (130, 130), (161, 160), (200, 190), (256, 256), (23, 23), (57, 57), (90, 90)]
    out = []
    for i, (m, n) in enumerate(shapes):
        G = np.asfortranarray(rng.standard_normal((m, n)))
        p = n if i == 3 else (0 if i == 5 else int(rng.integers(0, n + 1)))
        out.append((G, W.signs_random(rng, n, p)))
    return out


def _run(api, facs, **kw):
    dev = torch.device("cuda:0")
    Gs = [torch.from_numpy(G).to(dev).t().contiguous().t() for G, _ in facs]
    Js = [torch.from_numpy(J).to(dev) for _, J in facs]
    r = api.hsvd_solve_batched(Gs, Js, api.make_batch_opts(**kw), check=False)
    torch.cuda.synchronize()
    return r


def _check_factor(G, J, s, U, V, ref, tol_rel=1e-12):
    """sigma per sign group within max(tol_rel, u kappa_j) of the oracle,
    u kappa_j = u || |G| |v_j| || / sigma_j the change of sigma_j under a
    one-ulp componentwise perturbation of G (the floor below which no FP64
    method can pin a value); invariants to 1e-12 n."""
    m, n = G.shape
    kap = U64 * np.linalg.norm(np.abs(G) @ np.abs(ref["V"]), axis=0) / ref["sigma"]
    for sg in (1, -1):
        idx = np.where(J == sg)[0]
        if idx.size:
            o = np.argsort(ref["sigma"][idx])
            a, b = np.sort(s[idx]), ref["sigma"][idx][o]
            err = np.abs(a - b) / b / np.maximum(tol_rel, kap[idx][o])
            assert np.max(err) <= 1.0, (n, sg, np.max(err))
    assert np.max(np.abs(U.T @ U - np.eye(n))) <= 1e-12 * n
    Jd = np.diag(J.astype(float))
    assert np.max(np.abs(V.T @ Jd @ V - Jd)) / max(1.0, np.max(np.abs(V)) ** 2) <= 1e-12 * n
    res = np.linalg.norm(G @ V - U * s[None, :], axis=0) / (np.linalg.norm(G) * np.linalg.norm(V, axis=0))
    assert np.max(res) <= 1e-12 * n


def test_batched_matches_oracle(api):
    facs = _mixed()
    r = _run(api, facs)
    assert r.rc == api.HSVD_OK and all(st == 0 for st in r.status)
    assert r.info.kernel_launches == 1 and r.info.grid >= 1
    assert sum(r.info.resident) == len(facs)
    for k, (G, J) in enumerate(facs):
        ref = oracle.hsvd(G, J, G.shape[1] * U64, 30)
        assert ref["status"] == 0
        _check_factor(G, J, r.sigma[k].cpu().numpy(), r.U[k].cpu().numpy(), r.V[k].cpu().numpy(), ref)
        assert r.sweeps[k] <= ref["sweeps"] + 3


def test_batched_equals_single_pointwise_bitwise(api):
    facs = _mixed(12)[:10]
    r = _run(api, facs, group_width=1024)
    dev = torch.device("cuda:0")
    for k, (G, J) in enumerate(facs):
        one = api.hsvd_solve_ex(torch.from_numpy(G).to(dev), torch.from_numpy(J).to(dev),
                                api.make_opts(method=api.HSVD_METHOD_POINTWISE, sort=True,
                                              shorten=api.HSVD_SHORTEN_NEVER))
        assert one.status == 0 and one.sweeps == r.sweeps[k]
        assert torch.equal(one.sigma, r.sigma[k])
        assert torch.equal(one.U, r.U[k]) and torch.equal(one.V, r.V[k])


def test_group_widths_and_graph_are_bitwise_identical(api):
    facs = _mixed(13)
    runs = [_run(api, facs, group_width=w, use_graph=g) for w, g in ((1024, True), (512, True), (256, False))]
    for r in runs:
        assert r.rc == api.HSVD_OK
    # 256-thread groups with 55 KB of shared memory keep fewer factors resident
    assert runs[2].info.resident[0] < runs[0].info.resident[0]
    for k in range(len(facs)):
        for r in runs[1:]:
            assert torch.equal(runs[0].sigma[k], r.sigma[k])
            assert torch.equal(runs[0].V[k], r.V[k])
            assert r.sweeps[k] == runs[0].sweeps[k]


def test_cta_of_512_threads_is_bitwise_identical(api):
    """The 512-thread CTA (twice the registers a thread, no spills) runs the
    same per-factor code for groups of 512 and 256: the same bits as the
    1024-thread CTA at those widths; autotuned under it, widths stay <= 512."""
    facs = _mixed(14)
    for w in (512, 256):
        a = _run(api, facs, group_width=w)
        b = _run(api, facs, group_width=w, cta_threads=512)
        assert a.rc == b.rc == api.HSVD_OK
        assert a.info.cta_threads == 1024 and b.info.cta_threads == 512
        for k in range(len(facs)):
            assert torch.equal(a.sigma[k], b.sigma[k]) and torch.equal(a.V[k], b.V[k])
            assert a.sweeps[k] == b.sweeps[k]
    t = _run(api, facs, cta_threads=512)
    assert t.rc == api.HSVD_OK and all(w in (256, 512) for w in t.info.bucket_width)


def test_autotuner_runs_once_then_caches(api):
    facs = W.batch(300, nmin=16, nmax=120, seed=21)
    r1 = _run(api, facs)
    r2 = _run(api, facs)
    assert r1.rc == api.HSVD_OK and r2.rc == api.HSVD_OK
    assert r1.info.tuned in (1, 2) and r2.info.tuned == 2
    assert all(w in (256, 512, 1024) for w in r1.info.bucket_width)
    assert list(r1.info.bucket_width) == list(r2.info.bucket_width)
    for k in range(len(facs)):
        assert torch.equal(r1.sigma[k], r2.sigma[k])


def test_host_arrays_equal_device_arrays(api):
    facs = _mixed(14)[:8]
    rd = _run(api, facs, group_width=512)
    Gs = [torch.from_numpy(G) for G, _ in facs]
    Js = [torch.from_numpy(J) for _, J in facs]
    rh = api.hsvd_solve_batched(Gs, Js, api.make_batch_opts(group_width=512))
    assert rh.rc == api.HSVD_OK
    for k in range(len(facs)):
        assert torch.equal(rh.sigma[k], rd.sigma[k].cpu())
        assert torch.equal(rh.U[k], rd.U[k].cpu()) and torch.equal(rh.V[k], rd.V[k].cpu())


def test_per_factor_status(api):
    facs = _mixed(15)[:6]
    bad = facs[2][0].copy()
    bad[3, 4] = np.nan
    facs[2] = (bad, facs[2][1])
    r = _run(api, facs)
    assert r.status[2] == api.HSVD_ERR_NONFINITE
    assert r.rc == api.HSVD_ERR_NONFINITE
    assert all(r.status[k] == 0 for k in range(6) if k != 2)
    # a sweep cap of 1 leaves factors unconverged, with valid outputs
    r1 = _run(api, _mixed(15)[:4], max_sweeps=1)
    assert r1.rc == api.HSVD_NOT_CONVERGED and all(st == api.HSVD_NOT_CONVERGED for st in r1.status)


def test_empty_batch(api):
    r = api.hsvd_solve_batched([], [], check=False)
    assert r.rc == api.HSVD_OK


def test_full_size_batch_sampled_against_oracle(api):
    """The 10,000-factor workload (n uniform on [16, 256], m = n, random p) in
    the launch configuration the benchmark times; sampled factors against the
    oracle, every factor converged and satisfying U^T U = I."""
    facs = W.batch(10000, seed=4)
    r = _run(api, facs)
    assert r.rc == api.HSVD_OK and all(st == 0 for st in r.status)
    rng = np.random.default_rng(0)
    sample = sorted(rng.choice(len(facs), 6, replace=False).tolist()) + [int(np.argmax([G.shape[1] for G, _ in facs]))]
    for k in sample:
        G, J = facs[k]
        ref = oracle.hsvd(G, J, G.shape[1] * U64, 30)
        _check_factor(G, J, r.sigma[k].cpu().numpy(), r.U[k].cpu().numpy(), r.V[k].cpu().numpy(), ref)
    # orthogonality of every U (cheap on the GPU)
    worst = 0.0
    for k in range(0, len(facs), 7):
        U = r.U[k]
        n = U.shape[1]
        worst = max(worst, float((U.T @ U - torch.eye(n, dtype=U.dtype, device=U.device)).abs().max()) / n)
    assert worst <= 1e-12
