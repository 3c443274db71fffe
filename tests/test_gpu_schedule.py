"""The two sweep schedules of the blocked method (HSVD_SCHEDULE_STEPS: the
steps of the pivot strategy one after the other; HSVD_SCHEDULE_PAIRS: every
block-pair visit as a node of a dependency graph) perform the same arithmetic
on every visit, so their results agree bit for bit, in every form; both
agree with the oracle."""
import numpy as np
import pytest
import torch

import oracle
from paper_1008_1371_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_1008_1371_gb300 import api, build_lib

    build_lib.build()
    oracle.build()
    assert torch.cuda.is_available()
    return api


def _run(api, G, J, **kw):
    dev = torch.device("cuda:0")
    r = api.hsvd_solve_ex(torch.from_numpy(np.asfortranarray(G)).to(dev), torch.from_numpy(J).to(dev),
                          api.make_opts(**kw))
    torch.cuda.synchronize()
    return r


@pytest.mark.parametrize("b,n,m,prec", [(16, 200, 230, 0), (32, 256, 256, 0), (64, 384, 400, 0), (64, 320, 350, 1)])
def test_schedules_agree_bit_for_bit(api, b, n, m, prec):
    G, J = W.graded(n, m=m, decades=5.0, seed=61 + b)
    kw = dict(method=api.HSVD_METHOD_BLOCKED, block_w=b, precision=prec, max_sweeps=40)
    a = _run(api, G, J, schedule=api.HSVD_SCHEDULE_STEPS, **kw)
    p = _run(api, G, J, schedule=api.HSVD_SCHEDULE_PAIRS, **kw)
    assert a.status == p.status == api.HSVD_OK
    assert a.sweeps == p.sweeps and a.rotations == p.rotations and a.pair_updates == p.pair_updates
    assert torch.equal(a.sigma, p.sigma) and torch.equal(a.U, p.U) and torch.equal(a.V, p.V)
    ref = oracle.block_hsvd(G, J, b, n * 2.0 ** -53, 40, inner_mode=1, sort=False, want_u=False, want_v=False)
    s = p.sigma.cpu().numpy()
    for sg in (1, -1):
        x, y = np.sort(s[J == sg]), np.sort(ref["sigma"][J == sg])
        assert np.max(np.abs(x - y) / y) <= 1e-12


def test_schedules_with_learned_form_and_trace(api):
    """Masked sweeps (steps) and full sweeps (pairs) mix in the learned form;
    the training rows a plain solve exports are the same under both."""
    G, J = W.graded(256, seed=62)
    model = torch.zeros(api.HSVD_MLP_PARAMS, dtype=torch.float32, device="cuda")
    model[-1] = -4.0  # skip everything a mask may skip: judge sweeps do the work
    kw = dict(method=api.HSVD_METHOD_BLOCKED, block_w=16, sort=False, max_sweeps=60)
    a = _run(api, G, J, schedule=api.HSVD_SCHEDULE_STEPS, skip_model=model, **kw)
    p = _run(api, G, J, schedule=api.HSVD_SCHEDULE_PAIRS, skip_model=model, **kw)
    assert a.status == p.status == api.HSVD_OK and a.sweeps == p.sweeps
    assert torch.equal(a.sigma, p.sigma) and torch.equal(a.V, p.V)
    rows = []
    for sched in (api.HSVD_SCHEDULE_STEPS, api.HSVD_SCHEDULE_PAIRS):
        out = torch.zeros((16 * 8 * 30, api.HSVD_MLP_FEATURES + 1), dtype=torch.float32, device="cuda")
        r = _run(api, G, J, schedule=sched, trace_out=out, **kw)
        rows.append(out[:r.trace_rows].clone())
    assert rows[0].shape == rows[1].shape and torch.equal(rows[0], rows[1])


def test_schedules_with_a_partial_skip_mask(api):
    """A network that keeps some visits and skips others: under the pair
    schedule the mask stays on the device (skipped visits become empty
    kernels of one fixed graph), under the step schedule the host compacts
    the visit table.  Same visits kept, same bits, same counts."""
    from oracle import mlp as M

    G, J = W.graded(384, seed=64)
    # logit = 200 relu(f0) - 1, f0 = log2(max scaled |a_ij| / tol) / 64 from the
    # visit's last record: keep a visit whose block failed the test last time
    w = np.zeros(M.PARAMS, dtype=np.float32)
    w[M.OFF_W1 + 0] = 1.0
    w[M.OFF_W2 + 0] = 1.0
    w[M.OFF_W3 + 0] = 200.0
    w[M.OFF_B3] = -1.0
    p = torch.from_numpy(w).cuda()
    kw = dict(method=api.HSVD_METHOD_BLOCKED, block_w=16, sort=False, max_sweeps=80, skip_model=p)
    a = _run(api, G, J, schedule=api.HSVD_SCHEDULE_STEPS, **kw)
    q = _run(api, G, J, schedule=api.HSVD_SCHEDULE_PAIRS, **kw)
    plain = _run(api, G, J, method=api.HSVD_METHOD_BLOCKED, block_w=16, sort=False, max_sweeps=80)
    assert a.status == q.status == api.HSVD_OK
    assert (a.sweeps, a.masked_sweeps, a.judge_sweeps, a.pair_visits) == \
        (q.sweeps, q.masked_sweeps, q.judge_sweeps, q.pair_visits)
    nvis = (384 // 16) * (384 // 32)
    masked_visits = a.pair_visits - (a.sweeps - a.masked_sweeps) * nvis
    assert 0 < masked_visits < a.masked_sweeps * nvis  # the mask kept some visits and skipped others
    assert torch.equal(a.sigma, q.sigma) and torch.equal(a.V, q.V)
    s, r = q.sigma.cpu().numpy(), plain.sigma.cpu().numpy()
    for sg in (1, -1):
        x, y = np.sort(s[J == sg]), np.sort(r[J == sg])
        assert np.max(np.abs(x - y) / y) <= 1e-12


def test_pair_schedule_profile_and_early_stop(api):
    """Profiling under the pair schedule reports the sweeps' total only; the
    early stop behaves as under the step schedule."""
    G, J = W.gaussian(256, seed=63)
    kw = dict(method=api.HSVD_METHOD_BLOCKED, block_w=32, tol=2.0 ** -52, tstop=-1.0, max_sweeps=40)
    p = _run(api, G, J, schedule=api.HSVD_SCHEDULE_PAIRS, profile=True, **kw)
    a = _run(api, G, J, schedule=api.HSVD_SCHEDULE_STEPS, profile=True, **kw)
    assert p.status == a.status == api.HSVD_OK and p.stop_rule == a.stop_rule == api.HSVD_STOP_TANGENT
    assert p.sweeps == a.sweeps and torch.equal(p.sigma, a.sigma)
    assert p.ms_gram == p.ms_solve == p.ms_update == 0.0 and p.ms_other > 0.0
    assert a.ms_gram > 0.0 and a.ms_solve > 0.0 and a.ms_update > 0.0
