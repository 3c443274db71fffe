"""The C ABI library builds, loads without a GPU and exports every symbol the
header declares; host-only entry points (status strings, the pivot-strategy
table, argument checks) work on the CPU."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hsvd.h")


@pytest.fixture(scope="module")
def api():
    from paper_1008_1371_gb300 import api, build_lib

    build_lib.build()
    return api


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hsvd_[a-z_0-9]+)\s*\(", text)))


def test_header_symbols_exported(api):
    L = api.lib()
    names = _declared_functions()
    assert "hsvd_solve" in names and "hsvd_solve_ex" in names
    for name in names:
        assert hasattr(L, name), name  # ctypes resolves the symbol or raises


def test_status_strings(api):
    for code, name in ((0, "HSVD_OK"), (1, "HSVD_NOT_CONVERGED"), (-1, "HSVD_ERR_ARG"), (-2, "HSVD_ERR_RANK"),
                       (-3, "HSVD_ERR_NONFINITE"), (-4, "HSVD_ERR_CUDA"), (-5, "HSVD_ERR_NOMEM")):
        assert api.hsvd_status_string(code) == name
    assert api.hsvd_status_string(12345) == "HSVD_UNKNOWN_STATUS"


@pytest.mark.parametrize("r", [2, 4, 8, 16, 32, 64, 128, 256])
def test_library_strategy_matches_oracle_stepper(api, orc, r):
    """The library's closed-form modulus table and the oracle's Alg. 4.4
    stepper (written independently) give the same pair sets in every step,
    across two quasi-sweeps."""
    lib_t = api.hsvd_modulus_pairs(r, 2 * r)
    orc_t = orc.modulus_pairs(r, 2 * r)
    for s in range(2 * r):
        a = {tuple(sorted(p)) for p in lib_t[s].tolist()}
        b = {tuple(sorted(p)) for p in orc_t[s].tolist()}
        assert a == b, s
        # library slots are ordered by their smaller index, a < b inside a pair
        firsts = [p[0] for p in lib_t[s].tolist()]
        assert firsts == sorted(firsts) and all(p[0] < p[1] for p in lib_t[s].tolist())


def test_argument_errors_without_gpu(api):
    L = api.lib()
    G = np.zeros((4, 4))
    J = np.ones(4, dtype=np.int8)
    s = np.zeros(4)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    # a wide factor (m < n) with ldu < m, with ldv < n, with ldg < m; ldg < m; n < 1; bad pair-table argument
    U = np.zeros((4, 4))
    assert L.hsvd_solve(p(G), 3, 4, 4, p(J), 0.0, 30, p(s), p(U), 2, None, 4, None, None) == api.HSVD_ERR_ARG
    assert L.hsvd_solve(p(G), 3, 4, 4, p(J), 0.0, 30, p(s), None, 3, p(U), 3, None, None) == api.HSVD_ERR_ARG
    assert L.hsvd_solve(p(G), 3, 4, 2, p(J), 0.0, 30, p(s), None, 3, None, 4, None, None) == api.HSVD_ERR_ARG
    assert L.hsvd_solve(p(G), 4, 4, 3, p(J), 0.0, 30, p(s), None, 4, None, 4, None, None) == api.HSVD_ERR_ARG
    assert L.hsvd_solve(p(G), 4, 0, 4, p(J), 0.0, 30, p(s), None, 4, None, 4, None, None) == api.HSVD_ERR_ARG
    assert L.hsvd_solve(None, 4, 4, 4, p(J), 0.0, 30, p(s), None, 4, None, 4, None, None) == api.HSVD_ERR_ARG
    out = np.zeros(8, dtype=np.int32)
    assert L.hsvd_modulus_pairs(3, 1, p(out)) == api.HSVD_ERR_ARG
    o = api.make_opts(block_w=24)
    info = api.HsvdInfo()
    assert L.hsvd_solve_ex(p(G), 4, 4, 4, p(J), p(s), None, 4, None, 4, ctypes.byref(o), ctypes.byref(info),
                           None) == api.HSVD_ERR_ARG
    assert info.status == api.HSVD_ERR_ARG


def test_batched_argument_errors_without_gpu(api):
    L = api.lib()
    G = np.zeros((4, 4))
    J = np.ones(4, dtype=np.int8)
    s = np.zeros(4)
    arr = lambda *a: (ctypes.c_void_p * len(a))(*[x.ctypes.data for x in a])  # noqa: E731
    i64 = lambda *a: (ctypes.c_int64 * len(a))(*a)  # noqa: E731
    o = api.make_batch_opts()
    # negative count
    assert L.hsvd_solve_batched_ex(-1, None, None, None, None, None, None, None, None, None, None,
                                   ctypes.byref(o), None, None) == api.HSVD_ERR_ARG
    # m < n, then ldg < m
    assert L.hsvd_solve_batched_ex(1, arr(G), i64(3), i64(4), i64(4), arr(J), arr(s), None, None, None, None,
                                   ctypes.byref(o), None, None) == api.HSVD_ERR_ARG
    assert L.hsvd_solve_batched_ex(1, arr(G), i64(4), i64(4), i64(3), arr(J), arr(s), None, None, None, None,
                                   ctypes.byref(o), None, None) == api.HSVD_ERR_ARG
    # bad group width, reserved field set
    o2 = api.make_batch_opts(group_width=384)
    assert L.hsvd_solve_batched_ex(1, arr(G), i64(4), i64(4), i64(4), arr(J), arr(s), None, None, None, None,
                                   ctypes.byref(o2), None, None) == api.HSVD_ERR_ARG
    o3 = api.make_batch_opts()
    o3.reserved = 7
    assert L.hsvd_solve_batched_ex(1, arr(G), i64(4), i64(4), i64(4), arr(J), arr(s), None, None, None, None,
                                   ctypes.byref(o3), None, None) == api.HSVD_ERR_ARG
    # CTA size other than 512 / 1024, and a group wider than the 512-thread CTA
    for bad in (api.make_batch_opts(cta_threads=256), api.make_batch_opts(cta_threads=512, group_width=1024)):
        assert L.hsvd_solve_batched_ex(1, arr(G), i64(4), i64(4), i64(4), arr(J), arr(s), None, None, None, None,
                                       ctypes.byref(bad), None, None) == api.HSVD_ERR_ARG


def test_learned_option_errors_without_gpu(api):
    """The learned form and the trace export follow block-pair visits across
    sweeps: they need the blocked method without reordering; tau < 1."""
    L = api.lib()
    G = np.zeros((4, 4))
    J = np.ones(4, dtype=np.int8)
    s = np.zeros(4)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    model = np.zeros(api.HSVD_MLP_PARAMS, dtype=np.float32)
    info = api.HsvdInfo()
    for kw in (dict(method=api.HSVD_METHOD_POINTWISE), dict(method=api.HSVD_METHOD_BLOCKED, sort=True),
               dict(method=api.HSVD_METHOD_BLOCKED, sort=False, skip_tau=1.0)):
        o = api.make_opts(**kw)
        o.skip_model = model.ctypes.data
        assert L.hsvd_solve_ex(p(G), 4, 4, 4, p(J), p(s), None, 4, None, 4, ctypes.byref(o), ctypes.byref(info),
                               None) == api.HSVD_ERR_ARG, kw
    # a trace array with no room
    o = api.make_opts(method=api.HSVD_METHOD_BLOCKED, sort=False)
    o.trace_out = model.ctypes.data
    o.trace_cap = 0
    assert L.hsvd_solve_ex(p(G), 4, 4, 4, p(J), p(s), None, 4, None, 4, ctypes.byref(o), ctypes.byref(info),
                           None) == api.HSVD_ERR_ARG


def test_tstop_argument_errors_without_gpu(api):
    """The tangent threshold is 0 (off), negative (the paper's T_eps) or in
    (0, 1]; anything else is an argument error, found before any GPU work."""
    L = api.lib()
    G = np.zeros((4, 4))
    J = np.ones(4, dtype=np.int8)
    s = np.zeros(4)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    arr = lambda *a: (ctypes.c_void_p * len(a))(*[x.ctypes.data for x in a])  # noqa: E731
    i64 = lambda *a: (ctypes.c_int64 * len(a))(*a)  # noqa: E731
    info = api.HsvdInfo()
    for bad in (float("nan"), 1.5, float("inf")):
        o = api.make_opts(tstop=bad)
        assert L.hsvd_solve_ex(p(G), 4, 4, 4, p(J), p(s), None, 4, None, 4, ctypes.byref(o), ctypes.byref(info),
                               None) == api.HSVD_ERR_ARG, bad
        assert info.stop_rule == api.HSVD_STOP_NONE
        ob = api.make_batch_opts(tstop=bad)
        assert L.hsvd_solve_batched_ex(1, arr(G), i64(4), i64(4), i64(4), arr(J), arr(s), None, None, None, None,
                                       ctypes.byref(ob), None, None) == api.HSVD_ERR_ARG, bad
    assert api.HSVD_TSTOP_PAPER == 2.0 ** -26 / 2  # sqrt(2^-52) / 2


_LAYOUT_STRUCTS = {
    "hsvd_opts": "HsvdOpts",
    "hsvd_info": "HsvdInfo",
    "hsvd_batch_opts": "HsvdBatchOpts",
    "hsvd_batch_info": "HsvdBatchInfo",
}


def test_struct_layouts_match_header(api, tmp_path):
    """The ctypes mirrors of the option and report structs have the size and
    field offsets a C compiler gives the header's declarations."""
    import subprocess

    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "hsvd.h"', "int main(void) {"]
    for cname, pyname in _LAYOUT_STRUCTS.items():
        cls = getattr(api, pyname)
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for fname, _ in cls._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, fname, cname, fname))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(line.split()[:2]): int(line.split()[2]) for line in out if line.strip()}
    for cname, pyname in _LAYOUT_STRUCTS.items():
        cls = getattr(api, pyname)
        assert got[(cname, "size")] == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert got[(cname, fname)] == getattr(cls, fname).offset, (cname, fname)


def test_shorten_argument_errors_without_gpu(api):
    L = api.lib()
    G = np.zeros((6, 4))
    J = np.ones(4, dtype=np.int8)
    s = np.zeros(4)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    info = api.HsvdInfo()
    o = api.make_opts(shorten=3)
    assert L.hsvd_solve_ex(p(G), 6, 4, 6, p(J), p(s), None, 6, None, 4, ctypes.byref(o), ctypes.byref(info),
                           None) == api.HSVD_ERR_ARG
    R = np.zeros((4, 4))
    # m < n, ldg < m, ldr < n
    assert L.hsvd_shorten_qr(p(G), 3, 4, 6, p(R), 4, None, 6, None) == api.HSVD_ERR_ARG
    assert L.hsvd_shorten_qr(p(G), 6, 4, 5, p(R), 4, None, 6, None) == api.HSVD_ERR_ARG
    assert L.hsvd_shorten_qr(p(G), 6, 4, 6, p(R), 3, None, 6, None) == api.HSVD_ERR_ARG


def test_sym_argument_errors_without_gpu(api):
    """Host pointers and bad sizes are refused before any GPU work."""
    L = api.lib()
    M = np.eye(4)
    G = np.zeros((4, 4))
    J = np.zeros(4, dtype=np.int8)
    lam = np.zeros(4)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    assert L.hsvd_sym_factor(p(M), 4, 4, p(G), 4, p(J), None, None) == api.HSVD_ERR_ARG  # host arrays
    assert L.hsvd_sym_factor(p(M), 0, 4, p(G), 4, p(J), None, None) == api.HSVD_ERR_ARG
    assert L.hsvd_sym_factor(p(M), 4, 3, p(G), 4, p(J), None, None) == api.HSVD_ERR_ARG
    info = api.HsvdInfo()
    assert L.hsvd_sym_eig(p(M), 4, 4, p(lam), None, 4, None, ctypes.byref(info), None) == api.HSVD_ERR_ARG


def test_device_only_entries_refuse_host_pointers(api):
    """The entry points documented as device-only check every array they get
    and return HSVD_ERR_ARG for host memory, before any allocation or
    launch (a kernel handed a host pointer would fault instead).  Sizes are
    valid, so only the pointer kind trips the check."""
    L = api.lib()
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
    ERR = api.HSVD_ERR_ARG
    G = np.zeros((64, 32), order="F")
    R = np.zeros((32, 32), order="F")
    Q = np.zeros((64, 32), order="F")
    assert L.hsvd_shorten_qr(p(G), 64, 32, 64, p(R), 32, None, 64, None) == ERR
    assert L.hsvd_shorten_qr(p(G), 64, 32, 64, p(R), 32, p(Q), 64, None) == ERR
    col0 = np.array([0, 16], dtype=np.int32)
    A = np.zeros((32, 32))
    W = np.zeros((32, 32))
    sgn = np.ones(32, dtype=np.int8)
    rot = np.zeros(1, dtype=np.int32)
    assert L.hsvd_pivot_gram(p(G), 64, 64, 16, 1, p(col0), p(A), None) == ERR
    assert L.hsvd_pivot_solve(16, 1, p(A), p(sgn), 1e-14, 1, 1, p(W), p(rot), None, None) == ERR
    assert L.hsvd_pivot_update(p(G), 64, 64, 16, 1, p(col0), p(W), p(rot), None) == ERR
    Ax = np.zeros((128, 128))
    Wx = np.zeros((128, 128))
    col0x = np.array([0, 64], dtype=np.int32)
    assert L.hsvd_pivot_gram_x(p(G), 64, 64, 1, p(col0x), p(Ax), None) == ERR
    assert L.hsvd_pivot_update_x(p(G), 64, 64, 1, p(col0x), p(Wx), p(rot), None, None) == ERR
    prm = np.zeros(api.HSVD_MLP_PARAMS, dtype=np.float32)
    X = np.zeros(8, dtype=np.float32)
    y = np.zeros(1, dtype=np.float32)
    out = np.zeros(1, dtype=np.float32)
    grad = np.zeros_like(prm)
    assert L.hsvd_mlp_forward(p(prm), p(X), 1, p(out), None) == ERR
    assert L.hsvd_mlp_grad(p(prm), p(X), p(y), 1, p(grad), p(out), None) == ERR
    assert L.hsvd_mlp_adam(p(prm), p(np.zeros_like(prm)), p(np.zeros_like(prm)), p(grad), 1, 1e-3, 0.9, 0.999,
                           1e-8, None) == ERR
    c_p, i64 = ctypes.c_void_p, ctypes.c_int64
    L.hsvd_solve_pointwise_noalloc.argtypes = [c_p, i64, i64, i64, c_p, ctypes.c_double, ctypes.c_int,
                                               ctypes.c_int, c_p, c_p, i64, c_p, i64, c_p, c_p]
    L.hsvd_solve_pointwise_noalloc.restype = ctypes.c_int
    G4 = np.eye(4, order="F")
    J4 = np.ones(4, dtype=np.int8)
    s4 = np.zeros(4)
    assert L.hsvd_solve_pointwise_noalloc(p(G4), 4, 4, 4, p(J4), 0.0, 30, 1, p(s4), None, 4, None, 4, None,
                                          None) == ERR
