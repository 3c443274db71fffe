"""The allocation-free entry point, hsvd_solve_pointwise_noalloc.

Callers that cannot allocate device memory (another allocator owns the
device, allocation is forbidden after start-up, or the context is capped) use
this entry point: its scratch is a fixed array inside the library.  The test
calls it through the C ABI with device arrays, twice in a row on the same
scratch array, and checks each result against the allocating entry point
(hsvd_solve_ex with the pointwise method) within the tolerances of the other
GPU tests.  This file sorts last so a failure here leaves the rest of a
``-x`` run already done.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu
U64 = 2.0 ** -53


@pytest.fixture(scope="module")
def api():
    from paper_1008_1371_gb300 import api, build_lib

    build_lib.build()
    assert torch.cuda.is_available()
    L = api.lib()
    p, i64 = ctypes.c_void_p, ctypes.c_int64
    L.hsvd_solve_pointwise_noalloc.argtypes = [p, i64, i64, i64, p, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                               p, p, i64, p, i64, p, p]
    L.hsvd_solve_pointwise_noalloc.restype = ctypes.c_int
    return api


def _noalloc(api, G, J, tol, sort):
    m, n = G.shape
    dev = torch.device("cuda:0")
    Gd = torch.from_numpy(np.asfortranarray(G)).to(dev).t().contiguous().t()
    Jd = torch.from_numpy(J).to(dev)
    s = torch.empty(n, dtype=torch.float64, device=dev)
    U = torch.empty((n, m), dtype=torch.float64, device=dev).t()
    V = torch.empty((n, n), dtype=torch.float64, device=dev).t()
    sweeps = ctypes.c_int(0)
    stream = ctypes.c_void_p(torch.cuda.current_stream(dev).cuda_stream)
    st = api.lib().hsvd_solve_pointwise_noalloc(Gd.data_ptr(), m, n, Gd.stride(1), Jd.data_ptr(), tol, 30,
                                                1 if sort else 0, s.data_ptr(), U.data_ptr(), U.stride(1),
                                                V.data_ptr(), V.stride(1), ctypes.byref(sweeps), stream)
    torch.cuda.synchronize()
    return st, s.cpu().numpy(), U.cpu().numpy(), V.cpu().numpy(), sweeps.value


def _alloc(api, G, J, tol, sort):
    dev = torch.device("cuda:0")
    r = api.hsvd_solve_ex(torch.from_numpy(np.asfortranarray(G)).to(dev), torch.from_numpy(J).to(dev),
                          api.make_opts(tol=tol, max_sweeps=30, method=api.HSVD_METHOD_POINTWISE, sort=sort))
    torch.cuda.synchronize()
    return r.status, r.sigma.cpu().numpy(), r.U.cpu().numpy(), r.V.cpu().numpy(), r.sweeps


def test_noalloc_matches_allocating_entry_point_twice(api):
    from paper_1008_1371_gb300 import workloads

    # n = 156 is the largest square factor the limit allows: the scratch array
    # is then nearly full
    cases = [(workloads.gaussian(128, seed=1), True), (workloads.gaussian(37, m=50, p=11, seed=3), False),
             (workloads.gaussian(156, p=70, seed=4), True)]
    for (G, J), sort in cases:
        n = G.shape[1]
        tol = n * U64
        st_a, s_a, U_a, V_a, sw_a = _alloc(api, G, J, tol, sort)
        assert st_a == api.HSVD_OK
        for _ in range(2):  # two calls in a row share the same scratch array
            st, s, U, V, sw = _noalloc(api, G, J, tol, sort)
            assert st == api.HSVD_OK and sw == sw_a
            assert np.max(np.abs(s - s_a) / s_a) <= 1e-12
            assert np.max(np.abs(U - U_a)) <= 1e-12 * n
            assert np.max(np.abs(V - V_a)) <= 1e-12 * n * max(1.0, np.max(np.abs(V_a)))


@pytest.mark.parametrize("m,n", [(157, 157), (200, 200), (300, 150)])
def test_noalloc_rejects_sizes_beyond_its_limit(api, m, n):
    """n above HSVD_NOALLOC_MAX_N = 156, or a G too tall for one SM's shared
    memory: HSVD_ERR_ARG before anything is launched."""
    dev = torch.device("cuda:0")
    G = torch.zeros((n, m), dtype=torch.float64, device=dev).t()
    J = torch.ones(n, dtype=torch.int8, device=dev)
    s = torch.empty(n, dtype=torch.float64, device=dev)
    st = api.lib().hsvd_solve_pointwise_noalloc(G.data_ptr(), m, n, m, J.data_ptr(), 0.0, 30, 1, s.data_ptr(),
                                                None, m, None, n, None, None)
    assert st == api.HSVD_ERR_ARG
