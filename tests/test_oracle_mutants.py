"""The pins are strong enough to catch plausible mistakes in the oracle.

Each case plants one mistake (a dropped term, a flipped sign, a transposed
operand, a wrong index or threshold) in a temporary copy of the oracle's C
source, builds that copy with the same compiler flags, and runs a small
battery of the independent checks of ``test_oracle_pins.py`` against it: at
least one check must fail.  The unmodified source must pass the same battery.
Everything here runs on the CPU."""
import os
from fractions import Fraction

import numpy as np
import pytest

from paper_1008_1371_gb300 import workloads as W

U = 2.0 ** -53
SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "hsvd_oracle.c")

MUTANTS = {
    "hyperbolic_theta_sign": ("zeta = -(aii + ajj) / (2.0 * aij);", "zeta = (aii + ajj) / (2.0 * aij);"),
    "trig_zeta_swapped": ("zeta = (ajj - aii) / (2.0 * aij);", "zeta = (aii - ajj) / (2.0 * aij);"),
    "hyperbolic_cosh_as_cos": ("*c = orc_cosine(tt, 1, 1.0 / sqrt((1.0 - tt) * (1.0 + tt)));",
                               "*c = orc_cosine(tt, -1, 1.0 / sqrt(1.0 + tt * tt));"),
    "update_drops_hyp": ("    double ht = hyp < 0 ? -t : t;\n    for (int64_t i = 0; i < m; ++i) {",
                         "    double ht = t;\n    for (int64_t i = 0; i < m; ++i) {"),
    "update_operands_transposed": ("x[i] = fma(ht, yi, xi) * c;", "x[i] = fma(ht, xi, yi) * c;"),
    "dot_drops_first_term": ("for (int64_t i = 0; i < m; ++i) s += x[i] * y[i];",
                             "for (int64_t i = 1; i < m; ++i) s += x[i] * y[i];"),
    "stepper_threshold": ("if (ip[k] + jp[k] > r - 2) {", "if (ip[k] + jp[k] > r - 3) {"),
    "inner_diag_drops_hyp": ("A[p + (int64_t)p * nn] = fma(ht, apq, A[p + (int64_t)p * nn]);",
                             "A[p + (int64_t)p * nn] = fma(t, apq, A[p + (int64_t)p * nn]);"),
    "inner_update_transposed": ("const double np_ = fma(ht, axq, axp) * c;",
                                "const double np_ = fma(ht, axp, axq) * c;"),
    "inner_mirror_dropped": ("        A[p + (int64_t)x * nn] = np_;\n", ""),
    "inner_cross_pass_whole_triangle": ("for (int q = (mode == 1 ? h : p + 1); q < nn", "for (int q = p + 1; q < nn"),
    "inner_pass_skips_last_row": ("for (int p = 0; p < (mode == 1 ? h : nn - 1)", "for (int p = 0; p < (mode == 1 ? h : nn - 2)"),
    "inner_cross_shift_wrong": ("b = h + ((k + s) % h);", "b = h + ((k + 2 * s) % h);"),
    "block_update_transposed_W": ("* Wp[x + y * nn];", "* Wp[y + x * nn];"),
    "test_uses_product_not_sqrt": ("if (aij == 0.0 || fabs(aij) < tol * sqrt(aii * ajj)) return ORC_OK;",
                                   "if (aij == 0.0 || fabs(aij) < tol * (aii * ajj)) return ORC_OK;"),
    # the tangent-threshold stop (Sec. 2, Eq. 4.2)
    "conv_code_inverted": ("return (tstop > 0.0 && fabs(t) <= tstop) ? 1 : 3;",
                           "return (tstop > 0.0 && fabs(t) > tstop) ? 1 : 3;"),
    "conv_code_overwritten": ("*cd |= conv_code(t, tstop);", "*cd = conv_code(t, tstop);"),
    "block_code_overwritten": ("cd |= conv_code(tmax, tstop);", "cd = conv_code(tmax, tstop);"),
    "stop_on_large_tangents": ("if (cd == 0 || cd == 1) {", "if (cd == 0 || cd == 3) {"),
    "inner_tmax_first_rotation": ("if (fabs(t) > *tmax) *tmax = fabs(t);", "if (*tmax == 0.0) *tmax = fabs(t);"),
}


def _battery(orc, lib):
    """Returns the list of failed checks (empty when all hold)."""
    failed = []
    rng = np.random.default_rng(5)
    # closed-form root of the zeroing condition, exact rational arithmetic
    for hyp in (-1, 1):
        for _ in range(40):
            x, y = rng.standard_normal(4), rng.standard_normal(4) * 3
            aii, ajj, aij = float(x @ x), float(y @ y), float(x @ y)
            t, c, st = orc.rotation(aii, ajj, aij, hyp, lib=lib)
            F = Fraction
            res = F(aij) * (1 + hyp * F(t) ** 2) + F(t) * (F(aii) + hyp * F(ajj))
            sc = abs(F(aij)) * (1 + F(t) ** 2) + abs(F(t)) * (F(aii) + F(ajj))
            ok = st == 0 and abs(res) <= 8 * U * sc and abs(c - 1 / np.sqrt(1 - hyp * t * t)) <= 1e-15 * c
            if not ok:
                failed.append("rotation")
                break
    # strategy properties (Sec. 2): disjoint pairs, each pair once except
    # (i, i+4) twice, and the ninth step is the first with tasks reversed
    P = orc.modulus_pairs(8, 9, lib=lib)
    count = {}
    for s in range(8):
        if sorted(P[s].ravel().tolist()) != list(range(8)):
            failed.append("strategy")
            break
        for a, b in P[s]:
            count[(min(a, b), max(a, b))] = count.get((min(a, b), max(a, b)), 0) + 1
    want = {(i, j): (2 if j - i == 4 else 1) for i in range(8) for j in range(i + 1, 8)}
    if count != want or [sorted(p) for p in P[8]] != [sorted(p) for p in P[0]][::-1]:
        failed.append("strategy-cover")
    # pointwise: invariants and LAPACK eigenvalues of G J G^T
    n = 32
    G, J = W.gaussian(n, seed=7)
    Jd = np.diag(J.astype(float))
    for order in ("cyclic", "modulus"):
        r = orc.hsvd(G, J, n * U, 30, order=order, sort=True, lib=lib)
        if r["status"] != 0 or not np.all(np.isfinite(r["sigma"])):
            failed.append("pointwise-status-" + order)
            continue
        lam = np.sort(r["sigma"] ** 2 * J)
        ev = np.sort(np.linalg.eigvalsh((G * J[None, :]) @ G.T))
        if np.max(np.abs(lam - ev)) > 8 * n * U * np.max(np.abs(ev)):
            failed.append("pointwise-eig-" + order)
        V, Uo = r["V"], r["U"]
        if np.max(np.abs(V.T @ Jd @ V - Jd)) > 1e-12 * max(1, np.max(np.abs(V)) ** 2):
            failed.append("pointwise-junitary-" + order)
        if np.max(np.abs(G @ V - Uo * r["sigma"])) > 1e-12 * np.linalg.norm(G):
            failed.append("pointwise-residual-" + order)
    # scale invariance: sigma(alpha G) = alpha sigma(G), alpha a power of two
    r1 = orc.hsvd(G, J, n * U, 30, order="modulus", sort=True, lib=lib)
    r2 = orc.hsvd(G * 1024.0, J, n * U, 30, order="modulus", sort=True, lib=lib)
    if r1["status"] != 0 or r2["status"] != 0 or \
            np.max(np.abs(np.sort(r2["sigma"]) / 1024.0 - np.sort(r1["sigma"])) / np.sort(r1["sigma"])) > 1e-12:
        failed.append("scale")
    # the stopping test (Eq. 2.3) leaves the columns relatively orthogonal to tol
    for r in (r1, r2):
        if r["status"] == 0 and np.max(np.abs(r["U"].T @ r["U"] - np.eye(n))) > 2 * n * U + 8 * n * U:
            failed.append("final-orthogonality")
    # inner solve: congruence and eigenvalues of J A, in every mode and order
    nn = 16
    Gp = rng.standard_normal((40, nn))
    A = Gp.T @ Gp
    sg = W.signs_block(nn, 6)
    Jn = np.diag(sg.astype(float))
    ev = np.sort(np.linalg.eigvals(Jn @ A).real)
    for order in ("cyclic", "parallel"):
        for mode in (0, 1, 2):
            Ao, Wp, nrot, passes, st = orc.inner_solve(A, sg, nn * U, mode=mode, max_passes=20, order=order,
                                                       lib=lib)
            if st != 0 or not np.allclose(Wp.T @ A @ Wp, Ao, rtol=0, atol=1e-11 * np.max(np.abs(A))) \
                    or not np.allclose(np.sort(np.linalg.eigvals(Jn @ Ao).real), ev, rtol=1e-9) \
                    or np.max(np.abs(Wp.T @ Jn @ Wp - Jn)) > 1e-11 * max(1, np.max(np.abs(Wp)) ** 2):
                failed.append("inner-%s-%d" % (order, mode))
            elif mode == 0 and not np.allclose(np.sort(sg * np.diag(Ao)), ev, rtol=1e-9):
                failed.append("inner-diag-%s" % order)
            elif mode == 1 and nrot > (nn // 2) ** 2:
                failed.append("inner-cross-count-%s" % order)
        # a zero off-diagonal block: the cross pass is the identity
        Z = A.copy()
        Z[:8, 8:] = 0.0
        Z[8:, :8] = 0.0
        if orc.inner_solve(Z, sg, nn * U, mode=1, order=order, lib=lib)[2] != 0:
            failed.append("inner-cross-zero-%s" % order)
    # the hand-worked 4 x 4 blocks (two disjoint couplings, closed forms)
    for hyp, a, b, t, dd in ((-1, 2.0, 1.0, 1.0, (1.0, 3.0)), (1, 5.0, -4.0, 0.5, (3.0, 3.0))):
        B = np.array([[a, 0, b, 0], [0, a, 0, b], [b, 0, a, 0], [0, b, 0, a]])
        s4 = np.ones(4, dtype=np.int8) if hyp < 0 else np.array([1, 1, -1, -1], dtype=np.int8)
        c = 1 / np.sqrt(1 - hyp * t * t)
        for mode in (1, 2):
            Bo, Wb, nr, _, st = orc.inner_solve(B, s4, 4 * U, mode=mode, lib=lib)
            want = np.array([[c, 0, t * c, 0], [0, c, 0, t * c], [hyp * t * c, 0, c, 0], [0, hyp * t * c, 0, c]])
            if st != 0 or nr != 2 or np.max(np.abs(Wb - want)) > 8 * U or \
                    np.max(np.abs(Bo - np.diag([dd[0], dd[0], dd[1], dd[1]]))) > 64 * U:
                failed.append("inner-hand-%d-%d" % (hyp, mode))
    # every pair of the off-diagonal block is visited once per cross pass:
    # one coupling at (k, h + j) on a diagonal block is rotated exactly once
    D = np.diag(np.arange(1.0, nn + 1.0))
    for order in ("cyclic", "parallel"):
        for k, j in ((0, 1), (3, 6), (7, 2), (5, 5)):
            Dc = D.copy()
            Dc[k, 8 + j] = Dc[8 + j, k] = 0.3
            for mode in (1, 2):
                if orc.inner_solve(Dc, sg, nn * U, mode=mode, order=order, lib=lib)[2] != 1:
                    failed.append("inner-visit-%s-%d" % (order, mode))
    # one row-cyclic pass (Sec. 5): the pair visited last ends exactly zero
    # (or passes the test)
    Ab = Gp.T @ Gp * np.outer(10.0 ** -np.arange(nn) / 8, 10.0 ** -np.arange(nn) / 8)
    for mode, (p, q) in ((1, (7, 15)), (2, (14, 15))):
        Ao = orc.inner_solve(Ab, sg, nn * U, mode=mode, lib=lib)[0]
        if not (Ao[p, q] == 0.0 or abs(Ao[p, q]) < nn * U * np.sqrt(Ao[p, p] * Ao[q, q])):
            failed.append("inner-last-pair-%d" % mode)
    # blocked method against LAPACK
    r = orc.block_hsvd(G, J, 4, n * U, 30, inner_mode=1, lib=lib)
    lam = np.sort(r["sigma"] ** 2 * J)
    ev = np.sort(np.linalg.eigvalsh((G * J[None, :]) @ G.T))
    if r["status"] != 0 or np.max(np.abs(lam - ev)) > 8 * n * U * np.max(np.abs(ev)):
        failed.append("blocked")
    failed += _tstop_checks(orc, lib)
    return failed


def _tstop_checks(orc, lib):
    """The tangent-threshold pins of ``test_oracle_tstop.py`` in brief."""
    failed = []
    eps = 2.0 ** -52
    rng = np.random.default_rng(8)

    def solve(kind, G, J, tol, tstop, max_sweeps=40):
        if kind in ("cyclic", "modulus"):
            return orc.hsvd(G, J, tol, max_sweeps, order=kind, sort=kind == "modulus", tstop=tstop, lib=lib)
        return orc.block_hsvd(G, J, int(kind[5:]), tol, max_sweeps, inner_mode=1, sort=False, tstop=tstop, lib=lib)

    # one pair: the threshold is compared with the closed-form tangent
    for seed in range(4):
        G = np.asfortranarray(rng.standard_normal((3, 2)))
        J = np.array([1, 1 if seed % 2 else -1], dtype=np.int8)
        a = G.T @ G
        if J[0] == J[1]:
            t1 = np.tan(0.5 * np.arctan2(2 * abs(a[0, 1]), abs(a[0, 0] - a[1, 1])))
        else:
            t1 = np.tanh(0.5 * np.arctanh(2 * abs(a[0, 1]) / (a[0, 0] + a[1, 1])))
        for kind in ("cyclic", "modulus", "block1"):
            up, down = solve(kind, G, J, 2 * U, t1 * (1 + 1e-6)), solve(kind, G, J, 2 * U, t1 * (1 - 1e-6))
            if up["sweeps"] != 1 or up["stop"] != orc.ORC_STOP_TANGENT or down["sweeps"] < 2:
                failed.append("tstop-2x2-" + kind)
    # one large tangent early in a sweep keeps it going
    for hyp_a in (False, True):
        G = np.diag(np.arange(1.0, 17.0))
        G[0, 1], G[8, 9] = 0.7, 2e-9
        J = np.ones(16, dtype=np.int8)
        J[1] = -1 if hyp_a else 1
        for kind in ("cyclic", "modulus", "block4"):
            if solve(kind, np.asfortranarray(G), J, eps, orc.T_EPS)["sweeps"] < 2:
                failed.append("tstop-or-" + kind)
    # two rotations in one inner step, the small one first: the block's code
    # is its largest tangent's
    G = np.diag(np.arange(1.0, 17.0))
    G[0, 15], G[1, 14] = 2.5e-7, 5.0
    if solve("block4", np.asfortranarray(G), np.ones(16, dtype=np.int8), eps, orc.T_EPS)["sweeps"] < 2:
        failed.append("tstop-inner-max")
    # constructed ground truth at the paper's eps: the rule fires first and
    # the values hold to 1e-12; a vanishing threshold is the plain stop
    G, J, sig = W.paper(96, p=40, seed=77)
    for kind in ("cyclic", "modulus", "block8"):
        strict, early = solve(kind, G, J, eps, 0.0), solve(kind, G, J, eps, orc.T_EPS)
        tiny = solve(kind, G, J, eps, 1e-300)
        if early["status"] != 0 or early["stop"] != orc.ORC_STOP_TANGENT or early["sweeps"] >= strict["sweeps"]:
            failed.append("tstop-fires-" + kind)
        elif max(np.max(np.abs(np.sort(early["sigma"][J == s]) - np.sort(sig[J == s])) / np.sort(sig[J == s]))
                 for s in (1, -1)) > 1e-12:
            failed.append("tstop-truth-" + kind)
        if tiny["sweeps"] != strict["sweeps"] or not np.array_equal(tiny["sigma"], strict["sigma"]):
            failed.append("tstop-vanishing-" + kind)
    return failed


def _variant(orc, tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) >= 1, name
    path = tmp_path / ("orc_%s.c" % name)
    path.write_text(src.replace(old, new))
    so = orc.build(force=True, src=str(path), out=str(tmp_path / ("liborc_%s.so" % name)))
    return orc.load(so)


def test_battery_passes_on_oracle(orc):
    assert _battery(orc, orc.load()) == []


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_battery_catches_planted_mistake(orc, tmp_path, name):
    old, new = MUTANTS[name]
    lib = _variant(orc, tmp_path, name, old, new)
    assert _battery(orc, lib), "planted mistake %s went unnoticed" % name
