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


def test_model_two_by_two_is_the_oracle_bit_for_bit(orc, model):
    """One pair: one rotation, nothing for the two orders of rounding to
    differ on."""
    rng = np.random.default_rng(5)
    for hyp in (-1, 1):
        x, y = rng.standard_normal(5), rng.standard_normal(5)
        A = np.array([[x @ x, x @ y], [x @ y, y @ y]])
        sg = np.array([1, 1 if hyp < 0 else -1], dtype=np.int8)
        a = model.inner_solve(A, sg, 1e-15, mode=2)
        b = orc.inner_solve(A, sg, 1e-15, mode=2, order="parallel")
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[2] == b[2] == 1


def test_model_statuses(orc, model):
    """A hyperbolic pair with |zeta| <= 1 (equal columns of opposite sign) is
    rank deficiency in both; malformed orders are refused."""
    x = np.arange(1.0, 5.0)
    A = np.array([[x @ x, x @ x], [x @ x, x @ x]])
    sg = np.array([1, -1], dtype=np.int8)
    assert model.inner_solve(A, sg, 1e-15, mode=2)[4] == orc.ORC_RANK
    assert orc.inner_solve(A, sg, 1e-15, mode=2, order="parallel")[4] == orc.ORC_RANK
    assert model.inner_solve(np.eye(3), np.ones(3, dtype=np.int8), 1e-15)[4] == orc.ORC_ARG
