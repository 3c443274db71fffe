"""GB300-native one-sided Jacobi hyperbolic SVD.

The compute path is the CUDA library ``libhsvd.so`` (sources in ``csrc/``,
C ABI declared in ``include/hsvd.h``); ``api`` is its thin Python binding.
``workloads`` draws the seeded synthetic inputs.  Importing the package does
not load the CUDA library; the first use of an ``api`` function does, and
fails loudly if the library was not built.
"""
import importlib

__all__ = ["hsvd_solve", "hsvd_solve_ex", "hsvd_status_string", "workloads", "api"]


def __getattr__(name):
    if name in ("hsvd_solve", "hsvd_solve_ex", "hsvd_status_string"):
        return getattr(importlib.import_module(__name__ + ".api"), name)
    if name in ("api", "workloads", "build_lib"):
        return importlib.import_module(__name__ + "." + name)
    raise AttributeError(name)
