"""Writes the stored oracle values that the full-size parity tests and
bench.py's accuracy report compare with.  Calls only oracle/ (and the seeded
input generators).

Each file holds, per input column j, the oracle's sigma_j and its per-value
noise floor u || |G| |v_j| ||_2 / sigma_j (u = 2^-53): the first-order change
of sigma_j under a componentwise relative perturbation of G by one unit
roundoff, which no FP64 method can undercut.

  graded1024  G = B diag(10^(-6 i/n)), B i.i.d. N(0,1) (seed 2), n = 1024,
              J = diag(+1 x 512, -1 x 512): the row-cyclic oracle, one thread.
  graded8192  G = B diag(10^(-8 i/n)) (seed 5), n = 8192, J = diag(+1 x 4096,
              -1 x 4096): the modulus-parallel oracle (the disjoint pairs of
              each step on OpenMP threads; bit for bit the serial modulus
              order whatever the thread count).
  haar4096    G = Q1 diag(sigma) Q2 (seed 3), n = 4096, 2048 random +1 in J:
              the modulus-parallel oracle.

tol = n 2^-53 and at most 40 sweeps in every case.  The input generators
call the platform's libm and LAPACK, which may round differently on another
machine, so the header records a SHA-256 of the exact bytes of G; a reader
compares it with its own G before trusting the values (the Haar factor's QR
differs in the last bits between x86 and Arm hosts, so its file is written
on the machine that runs the GPU tests).

Usage: python tests/golden/make_golden.py [graded1024|graded8192|haar4096]
"""
import hashlib
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1008_1371_gb300 import workloads  # noqa: E402

U = 2.0 ** -53
CASES = {
    "graded1024": (lambda: workloads.graded(1024, decades=6.0, seed=2), "cyclic",
                   "graded 1024x1024 seed 2, J=+512/-512"),
    "graded8192": (lambda: workloads.graded(8192, decades=8.0, seed=5), "modulus",
                   "graded 8192x8192 (10^(-8i/n)) seed 5, J=+4096/-4096"),
    "haar4096": (lambda: workloads.haar(4096, seed=3), "modulus",
                 "Haar 4096x4096 sigma log-uniform [1e-6,1] seed 3, 2048 random +1 in J"),
}


def digest(G):
    return hashlib.sha256(np.ascontiguousarray(G, dtype="<f8").tobytes(order="F")).hexdigest()


def write(name):
    make, order, what = CASES[name]
    G, J = make()
    n = G.shape[1]
    threads = oracle.set_threads(0)
    t0 = time.time()
    r = oracle.hsvd(G, J, n * U, 40 if order == "modulus" else 30, order=order, want_u=False, want_v=True)
    dt = time.time() - t0
    assert r["status"] == 0, r["status"]
    kappa_u = U * np.linalg.norm(np.abs(G) @ np.abs(r["V"]), axis=0) / r["sigma"]
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), name + "_sigma.txt")
    mode = "row-cyclic" if order == "cyclic" else "modulus-parallel"
    tmp = out + ".tmp"
    np.savetxt(tmp, np.stack([r["sigma"], kappa_u], axis=1), fmt="%.17e",
               header="oracle %s sigma and u*kappa_j, %s, tol=n*2^-53, sweeps=%d\nsha256(G)=%s"
                      % (mode, what, r["sweeps"], digest(G)))
    os.replace(tmp, out)
    print(out, "sweeps", r["sweeps"], "threads", threads, "%.0f s" % dt, digest(G))


if __name__ == "__main__":
    for name in sys.argv[1:] or ["graded1024"]:
        write(name)
