"""CPU oracle for the one-sided Jacobi hyperbolic SVD.

Test infrastructure only: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` import it.  The library path never does; the two
share no code.  ``hsvd_oracle.c`` holds the arithmetic, ``oracle.py`` the
ctypes marshalling and its build step; ``mlp.py`` models the learned form's
network and ``split.py`` the split-precision Gram exactly, both in numpy;
``inner_model.c`` / ``inner_model.py`` model the library's inner-solve
kernels exactly (a model of the kernels, not the oracle).
"""
from .oracle import (  # noqa: F401
    ORC_ARG,
    ORC_NONFINITE,
    ORC_NOT_CONVERGED,
    ORC_OK,
    ORC_RANK,
    ORC_STOP_NONE,
    ORC_STOP_ORTHO,
    ORC_STOP_TANGENT,
    T_EPS,
    block_hsvd,
    build,
    hsvd,
    hyp_qr,
    hyp_qr_apply_tt,
    inner_solve,
    load,
    modulus_pairs,
    rotation,
    set_threads,
    sym_factor,
    wide_hsvd,
)
