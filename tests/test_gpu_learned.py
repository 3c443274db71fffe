"""The learned form: the network kernels against the CPU oracle
(oracle/mlp.py: float64 forward, backpropagation, Adam), the per-visit trace
and features against a CPU recomputation from the input factor, and the
masked solves against the plain blocked method and the CPU oracle (the
network may cost or save sweeps, never accuracy: the final sweep is always a
full plain one)."""
import numpy as np
import pytest
import torch

import oracle
from oracle import mlp as mlp_oracle
from paper_1008_1371_gb300 import workloads as W

pytestmark = pytest.mark.gpu
U64 = 2.0 ** -53
DEV = torch.device("cuda:0")


@pytest.fixture(scope="module")
def api():
    from paper_1008_1371_gb300 import api, build_lib

    build_lib.build()
    oracle.build()
    assert torch.cuda.is_available()
    return api


def _rand_params(seed, scale=0.3):
    return np.random.default_rng(seed).standard_normal(mlp_oracle.PARAMS).astype(np.float32) * scale


def _t(x):
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(DEV)


def test_mlp_forward_matches_oracle(api):
    rng = np.random.default_rng(1)
    p = _rand_params(2)
    X = rng.standard_normal((1000, 8)).astype(np.float32)
    got = api.hsvd_mlp_forward(_t(p), _t(X)).cpu().numpy().astype(np.float64)
    want = mlp_oracle.forward(p.astype(np.float64), X.astype(np.float64))
    assert np.max(np.abs(got - want) / (1.0 + np.abs(want))) <= 2e-5


@pytest.mark.parametrize("n", [1, 63, 64, 1000])
def test_mlp_grad_matches_oracle(api, n):
    rng = np.random.default_rng(n)
    p = _rand_params(3)
    X = rng.standard_normal((n, 8)).astype(np.float32)
    y = (rng.random(n) < 0.4).astype(np.float32)
    g, loss = api.hsvd_mlp_grad(_t(p), _t(X), _t(y))
    lw, gw = mlp_oracle.loss_grad(p.astype(np.float64), X.astype(np.float64), y.astype(np.float64))
    g = g.cpu().numpy().astype(np.float64)
    assert abs(float(loss.item()) - lw) <= 1e-5 * (1 + abs(lw))
    assert np.max(np.abs(g - gw)) <= 1e-4 * np.max(np.abs(gw)), np.max(np.abs(g - gw)) / np.max(np.abs(gw))
    # deterministic: the same call gives the same bits
    g2, _ = api.hsvd_mlp_grad(_t(p), _t(X), _t(y))
    assert np.array_equal(g2.cpu().numpy().astype(np.float64), g)


def test_adam_matches_oracle(api):
    rng = np.random.default_rng(4)
    p = rng.standard_normal(mlp_oracle.PARAMS).astype(np.float32)
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    pd, md, vd = _t(p), _t(m), _t(v)
    P, M, V = p.astype(np.float64), m.astype(np.float64), v.astype(np.float64)
    for t in range(1, 4):
        g = rng.standard_normal(mlp_oracle.PARAMS).astype(np.float32)
        api.hsvd_mlp_adam(pd, md, vd, _t(g), t, lr=1e-2)
        # the kernel's constants are FP32 numbers (0.999 becomes 0.99900001...)
        P, M, V = mlp_oracle.adam_step(P, M, V, g.astype(np.float64), t, lr=float(np.float32(1e-2)),
                                       b1=float(np.float32(0.9)), b2=float(np.float32(0.999)),
                                       eps=float(np.float32(1e-8)))
    assert np.max(np.abs(pd.cpu().numpy() - P)) <= 1e-6
    assert np.max(np.abs(vd.cpu().numpy() - V)) <= 1e-5 * np.max(np.abs(V))


def _solve(api, G, J, **kw):
    r = api.hsvd_solve_ex(torch.from_numpy(np.asfortranarray(G)).to(DEV), torch.from_numpy(J).to(DEV),
                          api.make_opts(method=api.HSVD_METHOD_BLOCKED, sort=False, **kw), check=False)
    torch.cuda.synchronize()
    return r


def test_trace_rows_and_first_step_features(api):
    """Rows of sweep 2 carry the features of the sweep-1 records; for the
    visits of step 0 of sweep 1 the pivot block is the Gram of the input, so
    the record is recomputed here from G."""
    n, b = 256, 32
    G, J = W.graded(n, decades=6.0, seed=31)
    nb = n // b
    nvis = nb * (nb // 2)
    out = torch.zeros((3 * nvis, 9), dtype=torch.float32, device=DEV)
    tol = n * U64
    r = _solve(api, G, J, block_w=b, max_sweeps=3, trace_out=out)
    assert r.trace_rows == 2 * nvis
    rows = out[:r.trace_rows].cpu().numpy().astype(np.float64)
    assert set(np.unique(rows[:, 8])) <= {0.0, 1.0}
    tab = api.hsvd_modulus_pairs(nb, 1)
    for k in range(nb // 2):
        I, Jb = int(tab[0][k][0]), int(tab[0][k][1])
        cols = np.r_[I * b:(I + 1) * b, Jb * b:(Jb + 1) * b]
        A = G[:, cols].T @ G[:, cols]
        rec = mlp_oracle.record(A, J[cols], b)
        _, _, rot, _, _ = oracle.inner_solve(A, J[cols], tol, mode=2, order="parallel")  # the kernel's pairs
        rec[2] = rot
        f = mlp_oracle.features(rec, 0, I, Jb, b, nb, 2, 3, tol)
        got = rows[k]
        for i in (0, 1, 4, 5, 6, 7):
            assert abs(got[i] - f[i]) <= 1e-5 * (1 + abs(f[i])), (k, i, got[i], f[i])
        assert abs(got[2] - f[2]) <= 0.05, (k, got[2], f[2])
        assert got[3] == pytest.approx(2.0 / 3)


def _model(b3, scale=0.0):
    p = np.zeros(mlp_oracle.PARAMS, dtype=np.float32)
    if scale:
        p[:] = np.random.default_rng(7).standard_normal(mlp_oracle.PARAMS) * scale
    p[mlp_oracle.OFF_B3] = b3
    return torch.from_numpy(p).to(DEV)


def test_never_skip_model_equals_plain_bitwise(api):
    G, J = W.graded(512, decades=6.0, seed=32)
    plain = _solve(api, G, J, block_w=32)
    lm = _solve(api, G, J, block_w=32, skip_model=_model(50.0))
    assert plain.status == 0 and lm.status == 0
    # sweeps 2.. run masked with every visit kept; the masked sweep without
    # rotations is followed by one full judge sweep
    assert lm.masked_sweeps == plain.sweeps - 1 and lm.judge_sweeps == 1 and lm.sweeps == plain.sweeps + 1
    assert torch.equal(plain.sigma, lm.sigma) and torch.equal(plain.V, lm.V)
    nvis = (512 // 32) * (512 // 64)
    assert lm.pair_visits == plain.pair_visits + nvis


def test_skip_everything_model_still_converges_to_plain(api):
    """Masked sweeps that skip every visit change nothing, and every full
    judge sweep repeats the plain method's sweep: the same bits at the end."""
    G, J = W.graded(512, decades=6.0, seed=33)
    plain = _solve(api, G, J, block_w=32)
    lm = _solve(api, G, J, block_w=32, skip_model=_model(-50.0), max_sweeps=60)
    assert lm.status == 0 and lm.judge_sweeps >= 1 and lm.masked_sweeps >= 1
    assert torch.equal(plain.sigma, lm.sigma) and torch.equal(plain.V, lm.V)
    assert lm.pair_visits == plain.pair_visits


@pytest.mark.parametrize("prec", [0, 1])
def test_random_model_keeps_accuracy(api, prec):
    n = 384
    G, J = W.graded(n, decades=6.0, seed=34)
    ref = oracle.hsvd(G, J, n * U64, 40)
    b = 64 if prec else 32
    lm = _solve(api, G, J, block_w=b, skip_model=_model(0.0, scale=0.5), max_sweeps=60, precision=prec)
    assert lm.status == 0
    s = lm.sigma.cpu().numpy()
    kap = U64 * np.linalg.norm(np.abs(G) @ np.abs(ref["V"]), axis=0) / ref["sigma"]
    for sg in (1, -1):
        idx = np.where(J == sg)[0]
        o = np.argsort(ref["sigma"][idx])
        err = np.abs(np.sort(s[idx]) - ref["sigma"][idx][o]) / ref["sigma"][idx][o]
        assert np.max(err / np.maximum(1e-12, kap[idx][o])) <= 1.0


def test_trained_network_saves_gram_work(api):
    """Train on traces of graded factors (other seeds), then solve a held-out
    graded factor with and without the network: same sigma, fewer Gram
    evaluations."""
    from paper_1008_1371_gb300 import learn

    train_set = [W.graded(512, decades=d, seed=s) for d, s in ((6.0, 101), (4.0, 102), (8.0, 103))]
    X, y = learn.collect(train_set, block_w=32)
    assert X.shape[0] > 1000 and 0.05 < float(y.mean()) < 0.95
    params, losses = learn.train(X, y, steps=300, lr=3e-3, batch=4096, seed=0)
    assert losses[-1] < losses[0]
    G, J = W.graded(512, decades=6.0, seed=104)
    plain = _solve(api, G, J, block_w=32)
    lm = _solve(api, G, J, block_w=32, skip_model=params, max_sweeps=60)
    assert plain.status == 0 and lm.status == 0
    rel = (lm.sigma - plain.sigma).abs() / plain.sigma
    assert float(rel.max()) <= 1e-11
    assert lm.pair_visits < plain.pair_visits, (lm.pair_visits, plain.pair_visits, lm.sweeps, plain.sweeps)


def _train_for(api, block, precision):
    from paper_1008_1371_gb300 import learn

    train_set = [W.graded(1024, decades=d, seed=s) for d, s in ((6.0, 100), (4.0, 101), (8.0, 102), (6.0, 103))]
    X, y = learn.collect(train_set, block_w=block, precision=precision)
    params, _ = learn.train(X, y, steps=600, lr=3e-3, batch=4096, seed=0)
    return params


def _timed(api, Gd, Jd, opts):
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    r = api.hsvd_solve_ex(Gd, Jd, opts)
    e1.record()
    e1.synchronize()
    return r, e0.elapsed_time(e1)


def _check_8192(api, Gd, Jd, J, r, ref_sigma, ref_floor):
    import golden_ref

    n = Gd.shape[1]
    assert r.status == 0
    golden_ref.assert_gate(J, r.sigma.cpu().numpy(), ref_sigma, ref_floor)
    I = torch.eye(n, dtype=torch.float64, device=DEV)
    assert float((r.U.T @ r.U - I).abs().max()) <= 1e-12 * n
    Jm = torch.diag(Jd.to(torch.float64))
    assert float((r.V.T @ Jm @ r.V - Jm).abs().max()) / max(1.0, float(r.V.abs().max()) ** 2) <= 1e-12 * n


@pytest.mark.parametrize("precision", [0, 1])
def test_full_size_graded8192_learned_vs_plain(api, precision):
    """The learned configuration at full size (graded 8192, condition 1e8,
    J = diag(+1 x 4096, -1 x 4096), b = 64), with FP64 products (the
    configuration as stated) and with split-precision products.  The network
    is trained by the library's kernels on traces of other graded factors.
    Plain and learned runs are each gated per value against the stored oracle
    values (the modulus-parallel CPU oracle on this factor,
    tests/golden/graded8192_sigma.txt) and satisfy the invariants of
    Eq. 1.1; the learned run ends with a full plain sweep, forms fewer
    Grams, and with FP64 products takes less time than the plain run (CUDA
    events; the training is outside both)."""
    import golden_ref

    params = _train_for(api, 64, precision)
    n = 8192
    G, J = W.graded(n, decades=8.0, seed=5)
    ref_sigma, ref_floor = golden_ref.load("graded8192", G)
    Gd = torch.from_numpy(np.asfortranarray(G)).to(DEV)
    Jd = torch.from_numpy(J).to(DEV)
    kw = dict(method=api.HSVD_METHOD_BLOCKED, block_w=64, sort=False, precision=precision)
    plain, plain_ms = _timed(api, Gd, Jd, api.make_opts(max_sweeps=40, **kw))
    _check_8192(api, Gd, Jd, J, plain, ref_sigma, ref_floor)
    s_plain = plain.sigma.clone()
    del plain
    lm, lm_ms = _timed(api, Gd, Jd, api.make_opts(max_sweeps=80, skip_model=params, **kw))
    _check_8192(api, Gd, Jd, J, lm, ref_sigma, ref_floor)
    assert lm.judge_sweeps >= 1
    rel = float(((lm.sigma - s_plain).abs() / s_plain).max())
    assert rel <= 1e-12, rel
    print("graded 8192 precision %d: plain %.0f ms, learned %.0f ms (%d masked + %d judge sweeps)"
          % (precision, plain_ms, lm_ms, lm.masked_sweeps, lm.judge_sweeps))
    if precision == 0:
        assert lm_ms < plain_ms, (lm_ms, plain_ms)
