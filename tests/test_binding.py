"""The Python binding refuses malformed arguments before it hands pointers to
the C ABI (a wrong size there would make a kernel read or write past a
buffer): signature length, preallocated outputs (shape, layout, dtype,
device), block-pair tables, network inputs.  Well-formed arguments pass the
checks and reach the library, which on a machine without a GPU answers with
an error status.  CPU only."""
import pytest
import torch


@pytest.fixture(scope="module")
def api():
    from paper_1008_1371_gb300 import api, build_lib

    build_lib.build()
    return api


def _colmajor(m, n):
    return torch.empty((n, m), dtype=torch.float64).t()


def _reaches_library(fn):
    """Calls fn; a ValueError means the binding refused the arguments."""
    from paper_1008_1371_gb300.api import HsvdError

    try:
        fn()
    except HsvdError:
        pass


def test_solve_outputs_checked(api):
    m, n = 12, 8
    G = torch.zeros((m, n), dtype=torch.float64)
    J = torch.ones(n, dtype=torch.int8)
    good = (torch.empty(n, dtype=torch.float64), _colmajor(m, n), _colmajor(n, n))
    _reaches_library(lambda: api.hsvd_solve_ex(G, J, out=good, check=False))
    _reaches_library(lambda: api.hsvd_solve_ex(G, J, out=(good[0], None, None), check=False))
    bad = {
        "short J": dict(J=torch.ones(n - 1, dtype=torch.int8)),
        "2-D J": dict(J=torch.ones((n, 1), dtype=torch.int8)),
        "short sigma": dict(out=(torch.empty(n - 1, dtype=torch.float64), good[1], good[2])),
        "float32 sigma": dict(out=(torch.empty(n, dtype=torch.float32), good[1], good[2])),
        "strided sigma": dict(out=(torch.empty(2 * n, dtype=torch.float64)[::2], good[1], good[2])),
        "U too small": dict(out=(good[0], _colmajor(m - 1, n), good[2])),
        "U row-major": dict(out=(good[0], torch.empty((m, n), dtype=torch.float64), good[2])),
        "V wrong shape": dict(out=(good[0], good[1], _colmajor(n, n - 1))),
        "V row-major": dict(out=(good[0], good[1], torch.empty((n, n), dtype=torch.float64))),
    }
    for what, kw in bad.items():
        args = dict(J=J, out=good)
        args.update(kw)
        with pytest.raises(ValueError):
            api.hsvd_solve_ex(G, args["J"], out=args["out"], check=False)
            pytest.fail(what)


def test_batched_outputs_checked(api):
    shapes = [(10, 6), (7, 7)]
    Gs = [torch.zeros(s, dtype=torch.float64) for s in shapes]
    Js = [torch.ones(s[1], dtype=torch.int8) for s in shapes]
    sig = [torch.empty(n, dtype=torch.float64) for _, n in shapes]
    Us = [_colmajor(m, n) for m, n in shapes]
    Vs = [_colmajor(n, n) for _, n in shapes]
    _reaches_library(lambda: api.hsvd_solve_batched(Gs, Js, out=(sig, Us, Vs), check=False))
    with pytest.raises(ValueError):  # a signature one short
        api.hsvd_solve_batched(Gs, [Js[0], Js[1][:-1]], check=False)
    with pytest.raises(ValueError):  # a U with a padded leading dimension
        padded = torch.empty((6, 12), dtype=torch.float64).t()[:10]
        api.hsvd_solve_batched(Gs, Js, out=(sig, [padded, Us[1]], Vs), check=False)
    with pytest.raises(ValueError):  # one V missing
        api.hsvd_solve_batched(Gs, Js, out=(sig, Us, Vs[:1]), check=False)


def test_symmetric_input_square(api):
    with pytest.raises(ValueError):
        api.hsvd_sym_factor(torch.zeros((5, 4), dtype=torch.float64))
    with pytest.raises(ValueError):
        api.hsvd_sym_eig(torch.zeros((4, 5), dtype=torch.float64))


def test_pivot_tables_checked(api):
    b = 16
    G = _colmajor(64, 4 * b)
    G.zero_()
    good = torch.tensor([[0, 2 * b], [b, 3 * b]], dtype=torch.int32)
    _reaches_library(lambda: api.hsvd_pivot_gram(G, b, good))
    for col0 in (torch.tensor([[0, 3 * b + 1]], dtype=torch.int32),   # block past the last column
                 torch.tensor([[-1, b]], dtype=torch.int32),
                 torch.tensor([0, b], dtype=torch.int32),             # not (npairs, 2)
                 torch.zeros((0, 2), dtype=torch.int32)):
        with pytest.raises(ValueError):
            api.hsvd_pivot_gram(G, b, col0)
    W = torch.zeros((2, 2 * b, 2 * b), dtype=torch.float64)
    rot = torch.ones(2, dtype=torch.int32)
    _reaches_library(lambda: api.hsvd_pivot_update(G, b, good, W, rot))
    with pytest.raises(ValueError):  # two pairs writing the same block
        api.hsvd_pivot_update(G, b, torch.tensor([[0, 2 * b], [2 * b, 3 * b]], dtype=torch.int32), W, rot)
    with pytest.raises(ValueError):  # the blocks of one pair overlap
        api.hsvd_pivot_gram(G, b, torch.tensor([[0, b // 2]], dtype=torch.int32))
    with pytest.raises(ValueError):
        api.hsvd_pivot_update(G, b, good, W[:1], rot)
    with pytest.raises(ValueError):
        api.hsvd_pivot_update(G, b, good, W, rot[:1])
    A = torch.zeros((2, 2 * b, 2 * b), dtype=torch.float64)
    sgn = torch.ones((2, 2 * b), dtype=torch.int8)
    _reaches_library(lambda: api.hsvd_pivot_solve(A, sgn, 1e-14))
    with pytest.raises(ValueError):
        api.hsvd_pivot_solve(A, sgn[:, :b], 1e-14)
    with pytest.raises(ValueError):
        api.hsvd_pivot_solve(torch.zeros((2, 24, 24), dtype=torch.float64), sgn, 1e-14)
    Gx = _colmajor(64, 256)
    Gx.zero_()
    gx = torch.tensor([[0, 128], [64, 192]], dtype=torch.int32)
    _reaches_library(lambda: api.hsvd_pivot_gram_x(Gx, gx))
    with pytest.raises(ValueError):
        api.hsvd_pivot_gram_x(Gx, torch.tensor([[0, 200]], dtype=torch.int32))
    Wx = torch.zeros((2, 128, 128), dtype=torch.float64)
    _reaches_library(lambda: api.hsvd_pivot_update_x(Gx, gx, Wx, rot))
    with pytest.raises(ValueError):
        api.hsvd_pivot_update_x(Gx, gx, Wx, rot, torch.zeros((2, 64), dtype=torch.int32))


def test_network_inputs_are_cuda_tensors(api):
    """The network kernels take CUDA float32 tensors only; host tensors are
    refused by the binding."""
    p = torch.zeros(api.HSVD_MLP_PARAMS, dtype=torch.float32)
    X = torch.zeros((4, api.HSVD_MLP_FEATURES), dtype=torch.float32)
    with pytest.raises(ValueError):
        api.hsvd_mlp_forward(p, X)
    with pytest.raises(ValueError):
        api.hsvd_mlp_grad(p, X, torch.zeros(4, dtype=torch.float32))
