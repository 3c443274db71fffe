"""Parity of the CUDA path with the CPU oracle, through the C ABI.

sigma: relative error <= 1e-12 per value against the oracle's row-cyclic
method (the benchmark spec's tolerance), compared per sign group after sorting
(the value assigned to a given column may legitimately differ between pivot
orders).  Invariants: max |U^T U - I|, max |V^T J V - J| / max(1, max|V|^2)
and max_j ||G v_j - sigma_j u_j|| / (||G||_F ||v_j||) <= 1e-12 n.  Singular
vectors: matched by sigma, equal up to sign.
"""
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


def _gpu(api, G, J, **kw):
    dev = torch.device("cuda:0")
    r = api.hsvd_solve_ex(torch.from_numpy(np.asfortranarray(G)).to(dev), torch.from_numpy(J).to(dev),
                          api.make_opts(**kw), check=False)
    torch.cuda.synchronize()
    out = dict(sigma=r.sigma.cpu().numpy(), status=r.status, sweeps=r.sweeps, method=r.method, rot=r.rotations,
               U=r.U.cpu().numpy() if r.U is not None else None, V=r.V.cpu().numpy() if r.V is not None else None)
    return out


def _sigma_err(J, a, b):
    err = 0.0
    for s in (1, -1):
        if np.any(J == s):
            x, y = np.sort(a[J == s]), np.sort(b[J == s])
            err = max(err, float(np.max(np.abs(x - y) / y)))
    return err


def _sigma_gate(G, J, got, ref, floor=1e-12):
    """Per-value gate: |sigma - sigma_oracle| / sigma_oracle <= max(floor, u kappa_j),
    u kappa_j = u || |G| |v_j| ||_2 / sigma_j the first-order change of sigma_j
    under a componentwise relative perturbation of G of one unit roundoff
    (delta sigma_j = u_j^T delta G v_j): a value that rounding G itself moves by
    more than `floor` cannot be pinned tighter by any FP64 method.  Returns the
    largest error / tolerance ratio and the number of values above `floor`."""
    kap = U64 * np.linalg.norm(np.abs(G) @ np.abs(ref["V"]), axis=0) / ref["sigma"]
    worst, loose = 0.0, 0
    for s in (1, -1):
        idx = np.where(J == s)[0]
        if idx.size == 0:
            continue
        order = np.argsort(ref["sigma"][idx])
        y = ref["sigma"][idx][order]
        tolj = np.maximum(floor, kap[idx][order])
        x = np.sort(got[idx])
        worst = max(worst, float(np.max(np.abs(x - y) / y / tolj)))
        loose += int(np.sum(tolj > floor))
    return worst, loose


def _invariants(G, J, r):
    n = G.shape[1]
    Jd = np.diag(J.astype(np.float64))
    U_, V, s = r["U"], r["V"], r["sigma"]
    orth = np.max(np.abs(U_.T @ U_ - np.eye(n)))
    junit = np.max(np.abs(V.T @ Jd @ V - Jd)) / max(1.0, np.max(np.abs(V)) ** 2)
    resid = np.max(np.linalg.norm(G @ V - U_ * s[None, :], axis=0)
                   / (np.linalg.norm(G) * np.linalg.norm(V, axis=0)))
    return orth, junit, resid


def _vectors_match(J, a, b, tol):
    """U (and V) columns of a and b agree up to sign, matched by sigma within
    each sign group (skipping clusters closer than 1e-8 relative)."""
    worst = 0.0
    for s in (1, -1):
        idx = np.where(J == s)[0]
        if idx.size == 0:
            continue
        ia = idx[np.argsort(a["sigma"][idx])]
        ib = idx[np.argsort(b["sigma"][idx])]
        sig = np.sort(a["sigma"][idx])
        gap = np.minimum(np.r_[np.inf, np.diff(sig)], np.r_[np.diff(sig), np.inf]) / sig
        for k in range(idx.size):
            if gap[k] < 1e-8:
                continue
            ua, ub = a["U"][:, ia[k]], b["U"][:, ib[k]]
            sgn = np.sign(ua @ ub)
            worst = max(worst, np.max(np.abs(ua - sgn * ub)))
            va, vb = a["V"][:, ia[k]], b["V"][:, ib[k]]
            worst = max(worst, np.max(np.abs(va - sgn * vb)) / max(1.0, np.max(np.abs(vb))))
    assert worst <= tol, worst


# ---------------------------------------------------------------- pointwise
def test_pointwise_gaussian_128(api):
    """128 x 128 N(0,1), J = diag(+1 x 64, -1 x 64), tol = 128 2^-53, 30 sweeps."""
    G, J = W.gaussian(128, seed=1)
    tol = 128 * U64
    ref = oracle.hsvd(G, J, tol, 30)
    r = _gpu(api, G, J, tol=tol, max_sweeps=30, method=api.HSVD_METHOD_POINTWISE)
    assert r["status"] == api.HSVD_OK and r["method"] == api.HSVD_METHOD_POINTWISE
    assert _sigma_err(J, r["sigma"], ref["sigma"]) <= 1e-12
    orth, junit, resid = _invariants(G, J, r)
    assert max(orth, junit, resid) <= 1e-12 * 128
    _vectors_match(J, r, ref, 1e-9)
    # same pivot order and sorting as the oracle's modulus mode
    ref2 = oracle.hsvd(G, J, tol, 30, order="modulus", sort=True)
    assert _sigma_err(J, r["sigma"], ref2["sigma"]) <= 1e-13
    assert abs(r["sweeps"] - ref2["sweeps"]) <= 1


@pytest.mark.parametrize("m,n,p,seed", [(1, 1, 1, 1), (3, 2, 1, 2), (37, 31, 10, 3), (300, 20, 20, 4),
                                        (64, 64, 0, 5), (65, 63, 63, 6), (130, 129, 64, 7)])
def test_pointwise_ragged(api, m, n, p, seed):
    G, J = W.gaussian(n, m=m, p=p, seed=seed)
    tol = max(n, 2) * U64
    ref = oracle.hsvd(G, J, tol, 40)
    r = _gpu(api, G, J, tol=tol, max_sweeps=40, method=api.HSVD_METHOD_POINTWISE)
    assert ref["status"] == 0 and r["status"] == api.HSVD_OK
    assert _sigma_err(J, r["sigma"], ref["sigma"]) <= 1e-12
    orth, junit, resid = _invariants(G, J, r)
    assert max(orth, junit, resid) <= 1e-12 * max(n, 2)


def test_pointwise_identity_signature_is_svd(api):
    G, _ = W.graded(96, decades=4, seed=9)
    J = np.ones(96, dtype=np.int8)
    r = _gpu(api, G, J, method=api.HSVD_METHOD_POINTWISE)
    ref = oracle.hsvd(G, J, 96 * U64, 30)
    assert r["status"] == 0
    assert _sigma_err(J, r["sigma"], ref["sigma"]) <= 1e-12
    sv = np.linalg.svd(G, compute_uv=False)
    assert np.max(np.abs(np.sort(r["sigma"])[::-1] - sv)) <= 4 * 96 * U64 * sv[0]


def test_pointwise_statuses(api):
    G, J = W.gaussian(16, seed=5)
    bad = G.copy()
    bad[2, 3] = np.inf
    assert _gpu(api, bad, J, method=api.HSVD_METHOD_POINTWISE)["status"] == api.HSVD_ERR_NONFINITE
    assert _gpu(api, G, J, max_sweeps=1, method=api.HSVD_METHOD_POINTWISE)["status"] == api.HSVD_NOT_CONVERGED
    Gr = np.asfortranarray(np.repeat(G[:, :1], 2, axis=1))
    assert _gpu(api, Gr, np.array([1, -1], dtype=np.int8),
                method=api.HSVD_METHOD_POINTWISE)["status"] == api.HSVD_ERR_RANK


# ---------------------------------------------------------------- blocked
@pytest.mark.parametrize("b,inner,sort", [(16, 0, False), (32, 0, False), (16, 1, False), (64, 0, False),
                                          (32, 1, False), (32, 0, True)])
def test_blocked_graded_256(api, b, inner, sort):
    n = 256
    G, J = W.graded(n, decades=6, seed=2)
    tol = n * U64
    ref = oracle.hsvd(G, J, tol, 40)
    r = _gpu(api, G, J, tol=tol, max_sweeps=40, method=api.HSVD_METHOD_BLOCKED, block_w=b, inner_mode=inner,
             sort=sort)
    assert r["status"] == api.HSVD_OK
    assert _sigma_err(J, r["sigma"], ref["sigma"]) <= 1e-12
    orth, junit, resid = _invariants(G, J, r)
    assert max(orth, junit, resid) <= 1e-12 * n
    _vectors_match(J, r, ref, 1e-8)
    # the oracle's blocked method with the same block width, inner mode and sorting
    # (the oracle numbers its inner modes 0 = full-block, 1 = block-oriented):
    # sigma against its row-cyclic inner order (Sec. 5), the sweep count
    # against its parallel inner order (the library's pairs)
    im = 1 if inner == api.HSVD_INNER_ORIENTED else 0
    ob = oracle.block_hsvd(G, J, b, tol, 40, inner_mode=im, inner_max_passes=8, sort=sort)
    assert ob["status"] == 0
    assert _sigma_err(J, r["sigma"], ob["sigma"]) <= 1e-12
    op = oracle.block_hsvd(G, J, b, tol, 40, inner_mode=im, inner_max_passes=8, sort=sort, inner_order="parallel",
                           want_u=False, want_v=False)
    assert op["status"] == 0 and abs(op["sweeps"] - r["sweeps"]) <= 1


@pytest.mark.parametrize("m,n,p,b", [(200, 100, 30, 16), (129, 97, 97, 16), (500, 130, 0, 32)])
def test_blocked_ragged(api, m, n, p, b):
    G, J = W.gaussian(n, m=m, p=p, seed=m + n)
    tol = n * U64
    ref = oracle.hsvd(G, J, tol, 40)
    r = _gpu(api, G, J, tol=tol, max_sweeps=40, method=api.HSVD_METHOD_BLOCKED, block_w=b)
    assert r["status"] == api.HSVD_OK
    assert _sigma_err(J, r["sigma"], ref["sigma"]) <= 1e-12
    orth, junit, resid = _invariants(G, J, r)
    assert max(orth, junit, resid) <= 1e-12 * n


def test_blocked_config_graded_1024(api):
    """The measured configuration: 1024 x 1024, G = B diag(10^(-6 i/n)),
    J = diag(+1 x 512, -1 x 512), b = 32; also with J = I."""
    n = 1024
    G, J = W.graded(n, decades=6, seed=2)
    tol = n * U64
    ref = oracle.hsvd(G, J, tol, 30)
    r = _gpu(api, G, J, tol=tol, max_sweeps=30, method=api.HSVD_METHOD_BLOCKED, block_w=32)
    assert r["status"] == api.HSVD_OK
    worst, loose = _sigma_gate(G, J, r["sigma"], ref)
    assert worst <= 1.0 and loose <= 4, (worst, loose)
    orth, junit, resid = _invariants(G, J, r)
    assert max(orth, junit, resid) <= 1e-12 * n
    Jp = np.ones(n, dtype=np.int8)
    r1 = _gpu(api, G, Jp, tol=tol, max_sweeps=30, method=api.HSVD_METHOD_BLOCKED, block_w=32)
    assert r1["status"] == api.HSVD_OK
    sv = np.linalg.svd(G, compute_uv=False)
    assert np.max(np.abs(np.sort(r1["sigma"])[::-1] - sv)) <= 4 * n * U64 * sv[0]
    orth, junit, resid = _invariants(G, Jp, r1)
    assert max(orth, junit, resid) <= 1e-12 * n


def test_blocked_statuses(api):
    G, J = W.gaussian(96, seed=8)
    bad = G.copy()
    bad[5, 7] = np.nan
    assert _gpu(api, bad, J, method=api.HSVD_METHOD_BLOCKED, block_w=16)["status"] == api.HSVD_ERR_NONFINITE
    r = _gpu(api, G, J, max_sweeps=1, method=api.HSVD_METHOD_BLOCKED, block_w=16)
    assert r["status"] == api.HSVD_NOT_CONVERGED and r["sweeps"] == 1


def test_deterministic_and_host_arrays(api):
    """Two calls give bitwise equal results; host (pinned) arrays give the same
    bits as device arrays."""
    G, J = W.graded(256, decades=6, seed=12)
    a = _gpu(api, G, J, method=api.HSVD_METHOD_BLOCKED, block_w=16)
    b = _gpu(api, G, J, method=api.HSVD_METHOD_BLOCKED, block_w=16)
    assert np.array_equal(a["sigma"], b["sigma"]) and np.array_equal(a["U"], b["U"])
    Gh = torch.from_numpy(np.asfortranarray(G)).pin_memory()
    Jh = torch.from_numpy(J).pin_memory()
    h = api.hsvd_solve_ex(Gh, Jh, api.make_opts(method=api.HSVD_METHOD_BLOCKED, block_w=16))
    assert h.status == 0 and h.sigma.device.type == "cpu"
    assert np.array_equal(h.sigma.numpy(), a["sigma"]) and np.array_equal(h.V.numpy(), a["V"])


# ---------------------------------------------------------------- kernels
@pytest.mark.parametrize("b", [16, 32, 64])
def test_kernel_gram(api, b):
    rng = np.random.default_rng(b)
    rows, ncols = 640, 8 * b
    G = rng.standard_normal((rows, ncols)) * 10.0 ** rng.uniform(-3, 3, ncols)[None, :]
    col0 = np.array([[0, 5 * b], [2 * b, 3 * b], [7 * b, 1 * b]], dtype=np.int32)
    dev = torch.device("cuda:0")
    A = api.hsvd_pivot_gram(torch.from_numpy(np.asfortranarray(G)).to(dev), b,
                            torch.from_numpy(col0).to(dev)).cpu().numpy()
    for k, (i0, j0) in enumerate(col0):
        P = np.concatenate([G[:, i0:i0 + b], G[:, j0:j0 + b]], axis=1)
        ref = P.T @ P
        bound = 2 * rows * U64 * (np.abs(P).T @ np.abs(P))
        assert np.all(np.abs(A[k] - ref) <= bound)
        assert np.array_equal(A[k], A[k].T)


def _pivot_blocks(b, seed, npairs=3):
    nn = 2 * b
    rng = np.random.default_rng(seed)
    As, sg = [], []
    for k in range(npairs):
        P = rng.standard_normal((3 * nn, nn)) * 10.0 ** rng.uniform(-3, 0, nn)[None, :]
        As.append(P.T @ P)
        sg.append(W.signs_block(nn, [nn // 2, 5, nn][k % 3]))
    return np.stack(As), np.stack(sg)


def _gpu_inner(api, As, sg, tol, mode, max_passes=10):
    dev = torch.device("cuda:0")
    Ao, Wg, rot, st = api.hsvd_pivot_solve(torch.from_numpy(As).to(dev), torch.from_numpy(sg).to(dev), tol,
                                           mode=mode, max_passes=max_passes)
    assert int(st.cpu()[0]) == 0
    return Ao.cpu().numpy(), Wg.cpu().numpy(), rot.cpu().numpy()


@pytest.mark.parametrize("b,mode", [(16, 0), (16, 1), (16, 2), (32, 0), (32, 1), (32, 2), (64, 1), (64, 2)])
def test_kernel_inner_solve_matches_model(api, b, mode):
    """Same A_P: the kernel reproduces the exact CPU model of its arithmetic
    (oracle/inner_model.c: the parallel strategy's pairs, a step's pairs at
    once, the halves of R^T A R alternating between steps) bit for bit (the
    library is compiled without floating-point contraction; every FMA is
    explicit on both sides)."""
    from oracle import inner_model

    nn = 2 * b
    As, sg = _pivot_blocks(b, 100 + b + mode)
    tol = nn * U64
    Ao, Wg, rot = _gpu_inner(api, As, sg, tol, mode)
    for k in range(As.shape[0]):
        Ar, Wr, nrot, passes, s = inner_model.inner_solve(As[k], sg[k], tol, mode=mode, max_passes=10)
        assert s == 0 and nrot == rot[k]
        assert np.array_equal(Wg[k], Wr), np.max(np.abs(Wg[k] - Wr))
        assert np.array_equal(Ao[k], Ar), np.max(np.abs(Ao[k] - Ar))


def _threshold_blocks(b, seed, npairs=3):
    """Pivot blocks whose off-diagonal entries sit on the threshold of Eq. 2.3,
    tol sqrt(a_ii a_jj) rounded as the test rounds it: exactly on it (the pair
    rotates), one ulp below (it passes), and 2^-14 .. 2^-20 to either side --
    inside and outside the margin within which the kernels' test falls back to
    the plain expression."""
    nn = 2 * b
    tol = nn * U64
    rng = np.random.default_rng(seed)
    As, sg = [], []
    rel = [0.0, -1.0, 2.0 ** -14, -(2.0 ** -14), 2.0 ** -17, -(2.0 ** -17), 2.0 ** -20, -(2.0 ** -20), 0.5, -0.5]
    for k in range(npairs):
        d = 10.0 ** rng.uniform(-4, 2, nn)
        A = np.diag(d)
        for x in range(nn):
            for y in range(x + 1, nn):
                T = tol * np.sqrt(d[x] * d[y])
                r = rel[rng.integers(len(rel))]
                v = np.nextafter(T, 0.0) if r == -1.0 else T * (1.0 + r)
                A[x, y] = A[y, x] = v * rng.choice([-1.0, 1.0])
        As.append(A)
        sg.append(W.signs_block(nn, [nn // 2, 5, nn][k % 3]))
    return np.stack(As), np.stack(sg)


@pytest.mark.parametrize("b,mode", [(16, 1), (16, 2), (64, 1), (64, 2), (32, 0)])
def test_kernel_threshold_pairs_match_model(api, b, mode):
    """Entries on the threshold of Eq. 2.3 (the kernels decide clear cases
    from exponents and single-precision mantissas and the rest with the plain
    expression; the model always uses the plain expression): kernel and
    model agree bit for bit, rotation counts included."""
    from oracle import inner_model

    nn = 2 * b
    As, sg = _threshold_blocks(b, 900 + b + mode)
    tol = nn * U64
    Ao, Wg, rot = _gpu_inner(api, As, sg, tol, mode)
    for k in range(As.shape[0]):
        Ar, Wr, nrot, passes, s = inner_model.inner_solve(As[k], sg[k], tol, mode=mode, max_passes=10)
        assert s == 0 and nrot == rot[k] and 0 < nrot
        assert np.array_equal(Wg[k], Wr), np.max(np.abs(Wg[k] - Wr))
        assert np.array_equal(Ao[k], Ar), np.max(np.abs(Ao[k] - Ar))


@pytest.mark.parametrize("b,mode", [(64, 0), (64, 1), (64, 2), (32, 0)])
def test_kernel_inner_solve_renormalising_blocks_match_model(api, b, mode):
    """Ungraded pivot blocks (P^T P, P standard normal): the large early
    rotations move the column scales of the scaled rotations out of
    [2^-8, 2^8] (at b = 64 the model renormalises five times in full-block mode
    and once in one full pass on these seeds), so the kernels' renormalisation
    is exercised; kernel and model agree bit for bit."""
    from oracle import inner_model

    nn = 2 * b
    rng = np.random.default_rng(7 + b)
    As, sg = [], []
    for trial in range(3):
        P = rng.standard_normal((nn, nn))
        As.append(P.T @ P)
        sg.append(W.signs_block(nn, [nn, nn // 2, 3][trial]))
    As, sg = np.stack(As), np.stack(sg)
    tol = nn * U64
    Ao, Wg, rot = _gpu_inner(api, As, sg, tol, mode)
    for k in range(As.shape[0]):
        Ar, Wr, nrot, passes, s = inner_model.inner_solve(As[k], sg[k], tol, mode=mode, max_passes=10)
        assert s == 0 and nrot == rot[k]
        assert np.array_equal(Wg[k], Wr), np.max(np.abs(Wg[k] - Wr))
        assert np.array_equal(Ao[k], Ar), np.max(np.abs(Ao[k] - Ar))


@pytest.mark.parametrize("b", [16, 32, 64])
def test_ring_full_pass_equals_transposing_pass(api, b):
    """The full pass on the ring of slots (mode 2, rows moving one slot per
    step between the CTAs of the cluster) and the transposing full pass
    (mode 0 stopped after one pass) apply the same rotations with the same
    element operations: A, W and the rotation counts agree bit for bit."""
    nn = 2 * b
    As, sg = _pivot_blocks(b, 300 + b, npairs=5)
    tol = nn * U64
    Ar, Wr, rr = _gpu_inner(api, As, sg, tol, 2)
    At, Wt, rt = _gpu_inner(api, As, sg, tol, 0, max_passes=1)
    assert np.array_equal(rr, rt)
    assert np.array_equal(Wr, Wt) and np.array_equal(Ar, At)


@pytest.mark.parametrize("b", [16, 64])
def test_ring_full_pass_rank_deficient_pair(api, b):
    """A hyperbolic pair with |zeta| <= 1 (two equal columns of opposite sign,
    every other pair already orthogonal) stops the pass at the first step that
    holds it with HSVD_ERR_RANK; A_P comes back as it stood (nothing rotated),
    from wherever the ring had moved its rows, as in the transposing pass."""
    nn = 2 * b
    dev = torch.device("cuda:0")
    rng = np.random.default_rng(b)
    A = np.diag(rng.uniform(1.0, 2.0, nn))
    p, q = 3, nn - 7  # a pair of a late step of the modulus order
    A[q, q] = A[p, p]
    A[p, q] = A[q, p] = A[p, p]
    sg = np.ones(nn, dtype=np.int8)
    sg[q] = -1
    out = []
    for mode, mp in ((2, 1), (0, 1)):
        Ao, Wg, rot, st = api.hsvd_pivot_solve(torch.from_numpy(A[None].copy()).to(dev),
                                               torch.from_numpy(sg[None].copy()).to(dev), nn * U64, mode=mode,
                                               max_passes=mp)
        assert int(st.cpu()[0]) == api.HSVD_ERR_RANK
        out.append((Ao.cpu().numpy()[0], Wg.cpu().numpy()[0], int(rot.cpu()[0])))
    (Ar, Wr, rr), (At, Wt, rt) = out
    assert rr == rt == 0
    assert np.array_equal(Ar, A) and np.array_equal(At, A)
    assert np.array_equal(Wr, np.eye(nn)) and np.array_equal(Wt, np.eye(nn))


@pytest.mark.parametrize("b,mode", [(16, 0), (16, 1), (16, 2), (32, 0), (32, 1), (32, 2), (64, 0), (64, 1), (64, 2)])
def test_kernel_inner_solve_against_oracle(api, b, mode):
    """The kernel against the oracle's plain inner solve (one rotation at a
    time as R^T A R) on the same A_P.
    - Same pairs (the oracle's parallel order): the same rotations are
      applied, only the rounding of entries that two rotations of a step
      both touch differs (about 3 roundings each, in another order), so per
      step the results differ by a few u of the entry's |R|^T |A| |R| scale;
      over a pass of at most 2b steps, carried through the later rotation
      parameters, the stated bound is |A_gpu - A_orc| <= 8 p (2b) u
      (|W|^T |A| |W|) and |W_gpu - W_orc| <= 8 p (2b) u max(1, max |W|), p the
      passes; the rotation counts agree.
    - The paper's row-cyclic order (Sec. 5) rotates other pairs in another
      order, so only what is order-free is compared: both are congruences by
      J-unitary W that keep the eigenvalues of J A, and in full-block mode
      both diagonals are those eigenvalues (per sign group)."""
    nn = 2 * b
    As, sg = _pivot_blocks(b, 200 + b + mode)
    tol = nn * U64
    Ao, Wg, rot = _gpu_inner(api, As, sg, tol, mode)
    for k in range(As.shape[0]):
        Ar, Wr, nrot, passes, s = oracle.inner_solve(As[k], sg[k], tol, mode=mode, max_passes=10, order="parallel")
        assert s == 0 and nrot == rot[k]
        bound = 8 * passes * nn * U64
        assert np.all(np.abs(Ao[k] - Ar) <= bound * (np.abs(Wr).T @ np.abs(As[k]) @ np.abs(Wr)))
        assert np.max(np.abs(Wg[k] - Wr)) <= bound * max(1.0, np.max(np.abs(Wr)))
        Jd = np.diag(sg[k].astype(float))
        ev = np.sort(np.linalg.eigvals(Jd @ As[k]).real)
        Ac, Wc, _, pc, s = oracle.inner_solve(As[k], sg[k], tol, mode=mode, max_passes=10, order="cyclic")
        assert s == 0
        for A_, W_ in ((Ao[k], Wg[k]), (Ac, Wc)):
            assert np.max(np.abs(W_.T @ Jd @ W_ - Jd)) <= 8 * max(pc, passes) * nn * U64 * max(1, np.max(np.abs(W_))) ** 2
            assert np.allclose(np.sort(np.linalg.eigvals(Jd @ A_).real), ev, rtol=1e-10, atol=0)
            if mode == 0:
                assert np.allclose(np.sort(sg[k] * np.diag(A_)), ev, rtol=1e-10, atol=0)


@pytest.mark.parametrize("b", [16, 32, 64])
@pytest.mark.parametrize("first", ["none", "late", "last"])
def test_kernel_cross_pass_late_first_rotation(api, b, first):
    """Cross pass (mode 1) on pivot blocks whose off-diagonal block is zero
    except at chosen pairs, so the first rotation comes at a chosen step (or
    never): the steps before it change nothing, and the kernel, which starts
    the pass at that step, still matches the exact model of its arithmetic bit
    for bit and rotates the same pairs as the oracle."""
    from oracle import inner_model

    nn, h = 2 * b, b
    rng = np.random.default_rng(500 + b)
    picks = {"none": [], "late": [(5, h // 2 + 1), (h - 2, h // 2 + 3)], "last": [(1, h - 1)]}[first]
    As, sg = [], []
    for k in range(3):
        A = np.zeros((nn, nn))
        for lo in (0, h):
            P = rng.standard_normal((2 * h, h)) * 10.0 ** rng.uniform(-2, 0, h)[None, :]
            A[lo:lo + h, lo:lo + h] = P.T @ P
        for i, s in picks:
            q = h + (i + s) % h
            A[i, q] = A[q, i] = 0.05 * np.sqrt(A[i, i] * A[q, q]) * (1 if k != 1 else -1)
        As.append(A)
        sg.append(W.signs_block(nn, [nn // 2, 5, nn][k]))
    As, sg = np.stack(As), np.stack(sg)
    dev = torch.device("cuda:0")
    tol = nn * U64
    Ao, Wg, rot, st = api.hsvd_pivot_solve(torch.from_numpy(As).to(dev), torch.from_numpy(sg).to(dev), tol, mode=1)
    Ao, Wg, rot = Ao.cpu().numpy(), Wg.cpu().numpy(), rot.cpu().numpy()
    assert int(st.cpu()[0]) == 0
    for k in range(3):
        Ar, Wr, nrot, passes, s = inner_model.inner_solve(As[k], sg[k], tol, mode=1)
        assert s == 0 and nrot == rot[k]
        assert np.array_equal(Wg[k], Wr) and np.array_equal(Ao[k], Ar)
        assert oracle.inner_solve(As[k], sg[k], tol, mode=1, order="parallel")[2] == nrot
        if first == "none":
            assert rot[k] == 0 and np.array_equal(Wg[k], np.eye(nn)) and np.array_equal(Ao[k], As[k])
        else:
            assert rot[k] >= len(picks)


@pytest.mark.parametrize("b", [16, 32, 64])
def test_kernel_update(api, b):
    nn = 2 * b
    rng = np.random.default_rng(7 * b)
    rows, ncols = 320, 6 * b
    X = rng.standard_normal((rows, ncols))
    col0 = np.array([[0, 3 * b], [4 * b, 1 * b], [2 * b, 5 * b]], dtype=np.int32)
    Wm = rng.standard_normal((3, nn, nn))
    rot = np.array([1, 0, 3], dtype=np.int32)
    dev = torch.device("cuda:0")
    Xd = torch.from_numpy(np.asfortranarray(X)).to(dev)
    Xd = Xd.t().contiguous().t()
    api.hsvd_pivot_update(Xd, b, torch.from_numpy(col0).to(dev), torch.from_numpy(Wm).to(dev),
                          torch.from_numpy(rot).to(dev))
    out = Xd.cpu().numpy()
    ref = X.copy()
    for k, (i0, j0) in enumerate(col0):
        if not rot[k]:
            continue
        cols = np.r_[i0:i0 + b, j0:j0 + b]
        ref[:, cols] = X[:, cols] @ Wm[k]
    err = np.max(np.abs(out - ref) / (np.abs(X).max() * np.abs(Wm).max() * nn))
    assert err <= 4 * nn * U64
    assert np.array_equal(out[:, 4 * b:5 * b], X[:, 4 * b:5 * b])  # pair 1 not rotated
