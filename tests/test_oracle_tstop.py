"""Pins for the oracle's tangent-threshold stop (Sec. 2: stop once every
computed tangent of a sweep is at most T_eps = sqrt(eps)/2; Eq. 4.2 gives the
convergence code of a rotation, (11)_2 if |t| > T_eps, (01)_2 otherwise, and
the codes are or-reduced over the sweep).  The checks rest on facts fixed
outside the oracle: the closed-form angle of a single pair, the bound |t| <= 1
of the smaller root, constructed ground truth, and the limit T -> 0 where the
rule must reduce to the plain stop.  No GPU needed."""
import numpy as np
import pytest

from paper_1008_1371_gb300 import workloads as W

U = 2.0 ** -53
EPS = 2.0 ** -52  # smallest power of two with fl(1 + eps) > 1 (Sec. 2)


def _tangent_2x2(G, J):
    """|t| of the one rotation that J-orthogonalises the two columns of G,
    from the angle itself: tan(2 phi) = 2 a_ij / (a_ii - a_jj) for equal signs,
    tanh(2 phi) = 2 a_ij / (a_ii + a_jj) for opposite signs; the smaller angle."""
    a = G.T @ G
    aii, ajj, aij = a[0, 0], a[1, 1], a[0, 1]
    if J[0] == J[1]:
        return np.tan(0.5 * np.arctan2(2.0 * abs(aij), abs(aii - ajj)))
    return np.tanh(0.5 * np.arctanh(2.0 * abs(aij) / (aii + ajj)))


def _solve(orc, kind, G, J, tol, max_sweeps=40, tstop=0.0, **kw):
    if kind == "cyclic":
        return orc.hsvd(G, J, tol, max_sweeps, order="cyclic", tstop=tstop, **kw)
    if kind == "modulus":
        return orc.hsvd(G, J, tol, max_sweeps, order="modulus", sort=True, tstop=tstop, **kw)
    b = int(kind[5:])  # "block<b>"
    return orc.block_hsvd(G, J, b, tol, max_sweeps, inner_mode=1, sort=False, tstop=tstop, **kw)


@pytest.mark.parametrize("kind", ["cyclic", "modulus", "block1"])
@pytest.mark.parametrize("seed", range(6))
def test_threshold_compares_the_tangent(orc, kind, seed):
    """One pair: the first sweep's largest tangent is the closed-form |t| of
    that pair (later rotations in the sweep are at rounding level).  A
    threshold just above it stops after sweep 1 with the tangent rule, one
    just below it does not."""
    rng = np.random.default_rng(300 + seed)
    G = np.asfortranarray(rng.standard_normal((3, 2)) * np.array([1.0, 10.0 ** rng.uniform(-1, 1)]))
    J = np.array([1, 1 if seed % 2 else -1], dtype=np.int8)
    t1 = _tangent_2x2(G, J)
    assert 1e-3 < t1 <= 1.0
    above = _solve(orc, kind, G, J, 2 * U, tstop=t1 * (1 + 1e-6))
    assert above["status"] == 0 and above["sweeps"] == 1 and above["stop"] == orc.ORC_STOP_TANGENT
    below = _solve(orc, kind, G, J, 2 * U, tstop=t1 * (1 - 1e-6))
    assert below["status"] == 0 and below["sweeps"] >= 2


def two_pair_factor(hyp_a):
    """16 x 16 factor whose columns are orthogonal except two pairs: A =
    (0, 1) with a large first tangent (closed form below) and B = (8, 9),
    in another block of width 4, with a tangent of about 1e-9 that still
    fails Eq. 2.3 at eps = 2^-52.  Every other pair is exactly orthogonal
    (disjoint supports), so nothing else ever rotates."""
    G = np.diag(np.arange(1.0, 17.0))
    G[0, 1] = 0.7
    G[8, 9] = 2e-9
    J = np.ones(16, dtype=np.int8)
    if hyp_a:
        J[1] = -1
    return np.asfortranarray(G), J


@pytest.mark.parametrize("kind", ["cyclic", "modulus", "block4"])
@pytest.mark.parametrize("hyp_a", [False, True])
def test_one_large_tangent_keeps_the_sweep_going(orc, kind, hyp_a):
    """A sweep with one rotation above the threshold cannot end the
    iteration, whatever rotates after it: the codes of Eq. 4.2 are or-ed over
    the whole sweep.  Pair A's first rotation uses the initial Gram entries
    (nothing else touches its columns first), so its tangent is the closed
    form; pair B's is far below T_eps."""
    G, J = two_pair_factor(hyp_a)
    tA = _tangent_2x2(G[:, :2], J[:2])
    tB = _tangent_2x2(G[:, 8:10], J[8:10])
    assert tA > 0.05 and tB < 0.2 * orc.T_EPS
    r = _solve(orc, kind, G, J, EPS, tstop=orc.T_EPS)
    assert r["status"] == 0 and r["sweeps"] >= 2
    ref = np.sort(np.abs(np.linalg.eigvals(np.diag(J.astype(float)) @ G.T @ G))) ** 0.5
    assert np.max(np.abs(np.sort(r["sigma"]) - ref) / ref) <= 1e-13


def test_block_code_takes_the_largest_inner_tangent(orc):
    """Blocked method, one pivot block (columns 0-3 and 12-15, b = 4) holding
    two non-orthogonal pairs that rotate in the same inner step: (0, 15)
    first with |t| about 1e-9, then (1, 14) with |t| about 0.04 (closed
    forms).  The block's code is that of its largest tangent, (11)_2, so the
    first sweep cannot end the iteration."""
    G = np.diag(np.arange(1.0, 17.0))
    G[0, 15] = 2.5e-7
    G[1, 14] = 5.0
    G = np.asfortranarray(G)
    J = np.ones(16, dtype=np.int8)
    small = _tangent_2x2(G[:, [0, 15]], J[[0, 15]])
    large = _tangent_2x2(G[:, [1, 14]], J[[1, 14]])
    assert small < 0.2 * orc.T_EPS and large > 0.01
    r = _solve(orc, "block4", G, J, EPS, tstop=orc.T_EPS)
    assert r["status"] == 0 and r["sweeps"] >= 2


@pytest.mark.parametrize("kind", ["cyclic", "modulus", "block4", "block8"])
def test_threshold_one_stops_after_first_sweep(orc, kind):
    """Every tangent is the smaller root, |t| <= 1 (tan of at most pi/4, or a
    tanh): with T = 1 the first sweep that rotates ends the iteration."""
    G, J = W.gaussian(48, seed=11)
    r = _solve(orc, kind, G, J, 48 * U, tstop=1.0)
    assert r["status"] == 0 and r["sweeps"] == 1 and r["stop"] == orc.ORC_STOP_TANGENT


@pytest.mark.parametrize("kind", ["cyclic", "modulus", "block4"])
def test_vanishing_threshold_is_the_plain_stop(orc, kind):
    """T -> 0: no tangent of a rotation is that small, so the rule never
    fires and the result is the plain one, bit for bit."""
    G, J = W.gaussian(40, seed=12)
    a = _solve(orc, kind, G, J, 40 * U)
    b = _solve(orc, kind, G, J, 40 * U, tstop=1e-300)
    assert a["status"] == b["status"] == 0
    assert a["stop"] == b["stop"] == orc.ORC_STOP_ORTHO
    assert a["sweeps"] == b["sweeps"] and a["rotations"] == b["rotations"]
    assert np.array_equal(a["sigma"], b["sigma"]) and np.array_equal(a["V"], b["V"])


@pytest.mark.parametrize("kind", ["modulus", "block8"])
def test_paper_threshold_ground_truth(orc, kind):
    """With eps of Eq. 2.3 at the paper's 2^-52 the threshold criterion
    ends the iteration first (Sec. 2 reports it always did), saving sweeps,
    and the values still match the constructed ground truth to 1e-12."""
    G, J, sig = W.paper(160, p=80, seed=220)
    strict = _solve(orc, kind, G, J, EPS)
    early = _solve(orc, kind, G, J, EPS, tstop=orc.T_EPS)
    assert strict["status"] == early["status"] == 0
    assert early["stop"] == orc.ORC_STOP_TANGENT and early["sweeps"] < strict["sweeps"]
    for s in (1, -1):
        got, ref = np.sort(early["sigma"][J == s]), np.sort(sig[J == s])
        assert np.max(np.abs(got - ref) / ref) <= 1e-12


def test_stop_is_a_truncation(orc):
    """The rule changes only where the iteration ends: the early result is
    the plain iteration's after the same number of sweeps, bit for bit."""
    G, J = W.graded(128, seed=5)
    early = _solve(orc, "modulus", G, J, EPS, tstop=orc.T_EPS)
    cut = _solve(orc, "modulus", G, J, EPS, max_sweeps=early["sweeps"])
    assert early["status"] == 0 and early["stop"] == orc.ORC_STOP_TANGENT
    assert cut["status"] == orc.ORC_NOT_CONVERGED
    assert np.array_equal(early["sigma"], cut["sigma"]) and np.array_equal(early["U"], cut["U"])


def test_sweeps_monotone_in_threshold(orc):
    """A larger threshold can only stop earlier."""
    G, J = W.gaussian(64, seed=13)
    counts = [_solve(orc, "modulus", G, J, 64 * U, tstop=T, want_u=False, want_v=False)["sweeps"]
              for T in (1e-300, 1e-12, 1e-9, orc.T_EPS, 1e-6, 1e-3, 0.1, 1.0)]
    assert all(x >= y for x, y in zip(counts, counts[1:])), counts
    assert counts[-1] == 1


def test_next_sweep_is_negligible(orc):
    """Eq. 2.6 with |t| <= T_eps: the diagonal moves by at most about eps/2
    of its size, so one more plain sweep after the stop changes no value by
    more than a few ulps (the reason the confirming sweep may be saved)."""
    G, J, _ = W.paper(96, p=10, seed=156)
    early = _solve(orc, "modulus", G, J, EPS, tstop=orc.T_EPS, want_u=False, want_v=False)
    more = _solve(orc, "modulus", G, J, EPS, max_sweeps=early["sweeps"] + 1, want_u=False, want_v=False)
    assert early["stop"] == orc.ORC_STOP_TANGENT
    assert np.max(np.abs(more["sigma"] - early["sigma"]) / early["sigma"]) <= 64 * U


def test_tstop_argument(orc):
    """A negative or NaN threshold is an argument error; T_eps = sqrt(2^-52)/2."""
    G, J = W.gaussian(8, seed=1)
    assert orc.hsvd(G, J, 8 * U, tstop=-1.0)["status"] == orc.ORC_ARG
    assert orc.block_hsvd(G, J, 2, 8 * U, tstop=float("nan"))["status"] == orc.ORC_ARG
    assert orc.T_EPS == np.sqrt(EPS) / 2
