"""Stored oracle values (written by tests/golden/make_golden.py, which calls
only the CPU oracle) and the per-value sigma gate of the full-size parity
tests."""
import hashlib
import os

import numpy as np

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load(name, G):
    """(sigma, u kappa_j) of the stored file `name`, after checking that it
    was computed for exactly these bytes of G."""
    path = os.path.join(HERE, "%s_sigma.txt" % name)
    assert os.path.exists(path), "no stored oracle values %s" % path
    head = [ln for ln in open(path) if ln.startswith("#")]
    want = head[1].split("sha256(G)=")[1].strip()
    have = hashlib.sha256(np.ascontiguousarray(G, dtype="<f8").tobytes(order="F")).hexdigest()
    assert want == have, "%s: the stored values belong to other bytes of G (this host's libm/LAPACK)" % name
    ref = np.loadtxt(path)
    return ref[:, 0], ref[:, 1]


def gate(J, sigma, ref_sigma, ref_floor):
    """Per sign group, sorted: |d sigma_j| / sigma_j against the oracle, over
    tol_j = max(1e-12, 2 u kappa_j).  u kappa_j (the floor) is the first-order
    change of sigma_j when G is rounded once, componentwise: the run and the
    oracle are two FP64 computations, each within about its floor of the exact
    value, so they may differ by twice it; where that is below 1e-12 the
    metric's 1e-12 applies.  Returns (the largest error / tol_j, the largest
    error among the values held to 1e-12, the floor of the value with the
    largest ratio, the number of values held to 2 u kappa_j)."""
    worst, worst_tight, floor_at, nloose = 0.0, 0.0, 0.0, 0
    for s in (1, -1):
        idx = np.where(J == s)[0]
        if idx.size == 0:
            continue
        o = np.argsort(ref_sigma[idx])
        y, k = ref_sigma[idx][o], ref_floor[idx][o]
        e = np.abs(np.sort(sigma[idx]) - y) / y
        tol = np.maximum(1e-12, 2.0 * k)
        r = e / tol
        i = int(np.argmax(r))
        if r[i] > worst:
            worst, floor_at = float(r[i]), float(k[i])
        tight = 2.0 * k <= 1e-12
        nloose += int((~tight).sum())
        if tight.any():
            worst_tight = max(worst_tight, float(e[tight].max()))
    return worst, worst_tight, floor_at, nloose


def assert_gate(J, sigma, ref_sigma, ref_floor):
    res = gate(J, sigma, ref_sigma, ref_floor)
    assert res[0] <= 1.0, "sigma beyond max(1e-12, 2 u kappa_j): ratio, tight max, floor there, loose count = %r" % (res,)
    return res
