"""fv_conserved_sums_noalloc: conservation sums for callers that cannot
allocate device memory (their device memory belongs to another allocator, or
their loop must not pay cudaMalloc's device-wide synchronisation).  Called
through the C ABI, it must return what fv_conserved_sums returns for the
same state -- bit for bit, the tolerance the sums tests use -- on two calls
in a row, whatever the previous call left in the shared scratch array.

Kept in a file that is collected last, so a run that stops at the first
failure has already run every other test."""
import ctypes

import numpy as np
import pytest

from paper_1812_07977_gb300 import problems

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    torch.cuda.set_device(0)
    from paper_1812_07977_gb300 import fv
    return fv.load_library()


def _noalloc(lib, U, l):
    out = (ctypes.c_double * 5)()
    _, nz, ny, nx = U.shape
    st = lib.fv_conserved_sums_noalloc(ctypes.c_void_p(U.data_ptr()), nx, ny, nz, l[0], l[1],
                                       l[2], ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                       out)
    assert st == 0, lib.fv_last_error().decode()
    return np.array(out[:])


def _with_mesh(U, l):
    from paper_1812_07977_gb300.fv import Mesh
    _, nz, ny, nx = U.shape
    with Mesh(nx, ny, nz, lx=l[0], ly=l[1], lz=l[2]) as m:
        m.set_state(U)
        return m.conserved_sums()


@pytest.mark.parametrize("shape,l", [((33, 17, 9), (1.0, 2.0, 0.5)),
                                     ((64, 48, 40), (1.0, 1.0, 1.0)),
                                     ((5, 3, 2), (0.3, 0.7, 1.1))])
def test_noalloc_sums_match_mesh_sums_twice(lib, shape, l):
    nx, ny, nz = shape
    first = torch.from_numpy(problems.random_smooth_periodic(nx, ny, nz, seed=41)).cuda()
    second = torch.from_numpy(problems.riemann_oblique(nx, ny, nz)).cuda()
    for U in (first, second):       # two calls in a row, different contents
        got = _noalloc(lib, U, l)
        ref = _with_mesh(U, l)
        assert np.array_equal(got, ref), (got, ref)
    # and the same state again after a different one
    assert np.array_equal(_noalloc(lib, first, l), _with_mesh(first, l))


def test_noalloc_sums_at_the_size_limit(lib):
    n = 256                          # 2^24 cells, the stated maximum
    U = torch.from_numpy(problems.riemann_oblique(n, n, n)).cuda()
    a = _noalloc(lib, U, (1.0, 1.0, 1.0))
    b = _noalloc(lib, U, (1.0, 1.0, 1.0))
    ref = _with_mesh(U, (1.0, 1.0, 1.0))
    assert np.array_equal(a, ref) and np.array_equal(b, ref)


def test_noalloc_rejects_sizes_beyond_the_limit(lib):
    U = torch.zeros((5, 1, 1, 8), dtype=torch.float64, device="cuda")
    out = (ctypes.c_double * 5)()
    st = lib.fv_conserved_sums_noalloc(ctypes.c_void_p(U.data_ptr()), 257, 256, 256, 1.0, 1.0,
                                       1.0, None, out)
    assert st == 1                   # FV_ERR_INVALID_ARG, before any device work
    assert "2^24" in lib.fv_last_error().decode()
    assert lib.fv_conserved_sums_noalloc(None, 4, 4, 4, 1.0, 1.0, 1.0, None, out) == 1
