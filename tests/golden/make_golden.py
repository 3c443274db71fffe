"""Writes the stored oracle values used by bench.py's accuracy report.

graded1024_sigma.txt: sigma (input column order) of the plain row-cyclic
FP64 oracle for G = B diag(10^(-6 i/n)), B i.i.d. N(0,1) (seed 2), n = 1024,
J = diag(+1 x 512, -1 x 512), tol = n 2^-53, plus the oracle's per-value
noise floor u || |G| |v_j| ||_2 / sigma_j.  Calls only oracle/.

The generator's libm calls may round differently on another machine, so the
header records a SHA-256 of the exact bytes of G; a reader compares it with
its own G before trusting the values.
"""
import os
import sys

import hashlib

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_1008_1371_gb300 import workloads  # noqa: E402

if __name__ == "__main__":
    n = 1024
    G, J = workloads.graded(n, decades=6.0, seed=2)
    r = oracle.hsvd(G, J, n * 2.0 ** -53, 30, want_u=False, want_v=True)
    assert r["status"] == 0, r["status"]
    kappa_u = 2.0 ** -53 * np.linalg.norm(np.abs(G) @ np.abs(r["V"]), axis=0) / r["sigma"]
    digest = hashlib.sha256(np.ascontiguousarray(G, dtype="<f8").tobytes(order="F")).hexdigest()
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "graded1024_sigma.txt")
    np.savetxt(out, np.stack([r["sigma"], kappa_u], axis=1), fmt="%.17e",
               header="oracle row-cyclic sigma and u*kappa_j, graded 1024x1024 seed 2, J=+512/-512, "
                      "tol=n*2^-53, sweeps=%d\nsha256(G)=%s" % (r["sweeps"], digest))
    print(out, r["sweeps"], digest)
