"""The exact model of the library's inner-solve kernels (oracle/inner_model.c)
against the oracle's plain inner solve, on the CPU.

The model applies the disjoint pairs of a step at once and alternates the two
halves of R^T A R between steps; the oracle applies one rotation at a time as
R^T A R.  With the oracle in the same (parallel) pair order the two apply the
same rotations: the rotation parameters of a step depend only on entries no
other pair of the step touches, so the rotation counts agree exactly, and only
the rounding of entries two rotations of a step both touch differs.  Per step
that is a few u of the entry's |R|^T |A| |R| scale; over a pass of at most 2b
steps, carried through the later rotation parameters, the stated bound is
|A_model - A_oracle| <= 8 p (2b) u (|W|^T |A| |W|) and |W_model - W_oracle| <=
8 p (2b) u max(1, max|W|), p the passes.  The GPU tests compare the kernels
with the model bit for bit and with the oracle within the same bound."""
import numpy as np
import pytest

from paper_1008_1371_gb300 import workloads as W

U = 2.0 ** -53


@pytest.fixture(scope="module")
def model(orc):
    from oracle import inner_model

    return inner_model


@pytest.mark.parametrize("nn", [2, 4, 16, 32, 64, 128])
@pytest.mark.parametrize("mode", [0, 1, 2])
def test_model_within_bound_of_oracle(orc, model, nn, mode):
    for seed in range(4):
        rng = np.random.default_rng(1000 * nn + 10 * mode + seed)
        P = rng.standard_normal((3 * nn, nn)) * 10.0 ** rng.uniform(-3, 0, nn)[None, :]
        A = P.T @ P
        sg = [W.signs_block(nn, nn // 2), W.signs_random(rng, nn, nn // 3), np.ones(nn, dtype=np.int8),
              -np.ones(nn, dtype=np.int8)][seed]
        tol = nn * U
        Am, Wm, nm, pm, sm = model.inner_solve(A, sg, tol, mode=mode, max_passes=10)
        Ao, Wo, no, po, so = orc.inner_solve(A, sg, tol, mode=mode, max_passes=10, order="parallel")
        assert sm == so == 0 and nm == no and pm == po
        bound = 8 * po * nn * U
        assert np.all(np.abs(Am - Ao) <= bound * (np.abs(Wo).T @ np.abs(A) @ np.abs(Wo)))
        assert np.max(np.abs(Wm - Wo)) <= bound * max(1.0, np.max(np.abs(Wo)))


def test_model_two_by_two_agrees_with_the_oracle(orc, model):
    """One pair: one rotation.  The model's (t, c) (reading M5) and the
    oracle's are two roundings of the same root, so the results agree to a
    few units in the last place."""
    rng = np.random.default_rng(5)
    for hyp in (-1, 1):
        for _ in range(20):
            x, y = rng.standard_normal(5), rng.standard_normal(5) * 10.0 ** rng.uniform(-3, 3)
            A = np.array([[x @ x, x @ y], [x @ y, y @ y]])
            sg = np.array([1, 1 if hyp < 0 else -1], dtype=np.int8)
            a = model.inner_solve(A, sg, 1e-15, mode=2)
            b = orc.inner_solve(A, sg, 1e-15, mode=2, order="parallel")
            if b[4] != 0:
                assert a[4] == b[4]
                continue
            assert a[2] == b[2] == 1
            scale = np.abs(b[1]).T @ np.abs(A) @ np.abs(b[1])
            assert np.all(np.abs(a[0] - b[0]) <= 16 * U * scale)
            assert np.max(np.abs(a[1] - b[1])) <= 16 * U * np.max(np.abs(b[1]))


def _exact_root(aii, ajj, aij, hyp):
    """The smaller root t of a_ij (t^2 + sg) + b t = 0 (Sec. 2), b rounded to
    double as the rotation forms it, to 60 digits."""
    from decimal import Decimal, getcontext

    getcontext().prec = 60
    b = Decimal(float(ajj - aii) if hyp < 0 else float(aii + ajj))
    zeta = (b if hyp < 0 else -b) / (2 * Decimal(float(aij)))
    r = (zeta * zeta + 1).sqrt() if hyp < 0 else (zeta * zeta - 1).sqrt()
    t = 1 / (abs(zeta) + r)
    return -t if zeta < 0 else t


def _cases(rng):
    """(a_ii, a_jj, a_ij, hyp): random magnitudes, equal diagonals, hyperbolic
    |zeta| on both sides of 2, ratios beyond 2^+-100, exponents beyond 2^+-800
    and a subnormal a_ij (the last three outside the single-precision start)."""
    out = []
    for _ in range(400):
        e = rng.uniform(-12, 12)
        aii, ajj = 10.0 ** (e + rng.uniform(-6, 6)), 10.0 ** (e + rng.uniform(-6, 6))
        aij = rng.choice([-1, 1]) * 10.0 ** (e + rng.uniform(-9, 3))
        out.append((aii, ajj, aij, -1))
        if abs(aii + ajj) > 2 * abs(aij):
            out.append((aii, ajj, aij, 1))
    for v in (1.0, 3.7e-9, 2.5e12):
        out += [(v, v, 0.3 * v, -1), (v, v, -1e-7 * v, -1), (v, v, 5e-40 * v, -1)]
        for zeta in (1.0000001, 1.5, 1.999999, 2.0, 2.000001, 2.5, 1e5, 1e7, 3e31):
            aij = -(2 * v) / (2 * zeta)
            out += [(v, v, aij, 1), (v, v, -aij, 1)]
    out += [(1.0, 2.0, 1e-33, -1), (1e-250, 3e-250, 1e-251, -1), (1e250, 3e250, 2e249, -1),
            (1.0, 1.5, 5e-310, -1), (2.0, 3.0, 1e-31, 1)]
    return out


def _single_precision_start(aii, ajj, aij, hyp):
    """Reading M5's range of the single-precision start, from the exponents."""
    b = (ajj - aii) if hyp < 0 else (aii + ajj)
    ea = np.frexp(aij)[1] - 1
    if abs(aij) < np.finfo(np.float64).tiny or not -800 < ea < 800:
        return False
    if b == 0.0:
        return hyp < 0
    eb = np.frexp(b)[1] - 1
    if abs(b) < np.finfo(np.float64).tiny or abs(eb - ea) > 100:
        return False
    return hyp < 0 or abs(b) >= 4 * abs(aij)


def test_model_rotation_pinned_to_the_exact_root(orc, model):
    """Reading M5 against the mathematics.  In the range of the
    single-precision start: t within 4 units in the last place of the exact
    smaller root (for the double b the rotation forms), and c consistent with
    that t to 4 u: |c sqrt(1 - hyp t^2) - 1| <= 4 u, and q the reciprocal of
    c to rounding, |c q - 1| <= 1.5 u with a mean below 0.15 u (the running
    column scales of the inner solve multiply by c and by q, so a bias of
    c q - 1 would add up over a visit) -- the J-orthogonality of the applied
    rotation rests on these.  Outside it: the oracle's t and c bit for bit,
    q again the reciprocal of c to rounding."""
    from decimal import Decimal, getcontext

    getcontext().prec = 60
    rng = np.random.default_rng(11)
    nfast, cq_sum = 0, Decimal(0)
    for aii, ajj, aij, hyp in _cases(rng):
        t, c, q, st = model.rotation(aii, ajj, aij, hyp)
        assert st == 0, (aii, ajj, aij, hyp)
        if not _single_precision_start(aii, ajj, aij, hyp):
            to, co, so = orc.rotation(aii, ajj, aij, hyp)
            assert so == 0 and t == to and c == co
            assert abs(Decimal(c) * Decimal(q) - 1) <= Decimal(1.5 * U)
            continue
        nfast += 1
        te = _exact_root(aii, ajj, aij, hyp)
        assert abs(Decimal(t) - te) <= 4 * Decimal(float(np.spacing(abs(float(te))))), (aii, ajj, aij, hyp, t, te)
        x = 1 + Decimal(t) * Decimal(t) if hyp < 0 else 1 - Decimal(t) * Decimal(t)
        assert abs(Decimal(c) * x.sqrt() - 1) <= 4 * Decimal(U), (aii, ajj, aij, hyp, c)
        cq = Decimal(c) * Decimal(q) - 1
        assert abs(cq) <= Decimal(1.5 * U), (aii, ajj, aij, hyp, q)
        cq_sum += cq
    assert nfast > 500
    assert abs(cq_sum / nfast) <= Decimal(0.15 * U)


def test_model_rotation_rank_deficiency_is_the_oracles(orc, model):
    """A hyperbolic pair with |zeta| <= 1 has no rotation in either; just
    above 1 both rotate."""
    for v, zeta in ((1.0, 1.0), (2.0, 0.5), (3.0, 1.0 + 2 ** -40)):
        aij = -(2 * v) / (2 * zeta)
        m = model.rotation(v, v, aij, 1)
        o = orc.rotation(v, v, aij, 1)
        assert (m[3] != 0) == (o[2] != 0) == (zeta <= 1.0)


def test_model_statuses(orc, model):
    """A hyperbolic pair with |zeta| <= 1 (equal columns of opposite sign) is
    rank deficiency in both; malformed orders are refused."""
    x = np.arange(1.0, 5.0)
    A = np.array([[x @ x, x @ x], [x @ x, x @ x]])
    sg = np.array([1, -1], dtype=np.int8)
    assert model.inner_solve(A, sg, 1e-15, mode=2)[4] == orc.ORC_RANK
    assert orc.inner_solve(A, sg, 1e-15, mode=2, order="parallel")[4] == orc.ORC_RANK
    assert model.inner_solve(np.eye(3), np.ones(3, dtype=np.int8), 1e-15)[4] == orc.ORC_ARG
