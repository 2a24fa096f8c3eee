"""The allocation-free gamma entry point (gnp_gamma_noalloc) on the GPU.

It serves callers that must not allocate device memory when they call in (applications
whose device memory belongs to their own pool or arena, plug-ins that receive only a
stream and their host's buffers, loops that cannot take cudaMalloc's synchronisation):
all its scratch is a fixed device array inside the library.  Checked through the C ABI
against gnp_gamma (which builds a gnp_mat and allocates) on two calls in a row with
different matrices, so the second call also shows that the shared scratch is cleared
between calls; an oversize n is refused with a clear message; a malformed CSR (a column
index equal to n, decreasing row pointers, row pointers that do not end at nnz) gives
NaN, every access of the kernel staying inside the buffers the sizes describe.  This
file is collected last so that a run stopping at the first failure has run every other
test.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2406_00809_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-13  # the relative tolerance of the gamma parity tests


@pytest.fixture(scope="module")
def gnp():
    import torch
    from paper_2406_00809_gb300 import build, gnp as g
    build.build()
    assert torch.cuda.is_available()
    return g


def _dev(a, dtype):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def test_gamma_noalloc_matches_gamma_on_two_calls(gnp):
    import torch
    lib = gnp.lib()
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    for A in (I.convdiff2d(64, 100.0), I.powerlaw(20_000, seed=9)):
        rp, col, val = _dev(A.row_ptr, torch.int32), _dev(A.col, torch.int32), _dev(A.val, torch.float64)
        st = lib.gnp_gamma_noalloc(A.n, A.nnz, C.c_void_p(rp.data_ptr()), C.c_void_p(col.data_ptr()),
                                   C.c_void_p(val.data_ptr()), C.c_void_p(out.data_ptr()),
                                   gnp._stream(None))
        assert st == 0, lib.gnp_last_error()
        torch.cuda.synchronize()
        ref = gnp.gnp_gamma(gnp.mat_from_csr(A))
        assert abs(out.item() - ref) <= TOL * ref, (out.item(), ref)


def test_gamma_noalloc_refuses_oversize(gnp):
    import torch
    lib = gnp.lib()
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    rp = torch.zeros(2, dtype=torch.int32, device="cuda")
    st = lib.gnp_gamma_noalloc((1 << 20) + 1, 0, C.c_void_p(rp.data_ptr()), None, None,
                               C.c_void_p(out.data_ptr()), gnp._stream(None))
    assert st == 1
    assert b"fixed scratch" in lib.gnp_last_error()


def _noalloc(gnp, n, nnz, rp, col, val, out):
    lib = gnp.lib()
    return lib.gnp_gamma_noalloc(n, nnz, C.c_void_p(rp.data_ptr()), C.c_void_p(col.data_ptr()),
                                 C.c_void_p(val.data_ptr()), C.c_void_p(out.data_ptr()), gnp._stream(None))


def test_gamma_noalloc_malformed_csr_gives_nan(gnp):
    import torch
    A = I.poisson2d(8)
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    val = _dev(A.val, torch.float64)
    cases = []
    col = A.col.copy()
    col[5] = A.n                       # a column index outside [0, n)
    cases.append((A.row_ptr, col))
    rp = A.row_ptr.copy()
    rp[3], rp[4] = rp[4], rp[3]        # decreasing row pointers (still inside [0, nnz])
    cases.append((rp, A.col))
    rp = A.row_ptr.copy()
    rp[-1] = A.nnz - 2                 # the last row pointer is not nnz
    cases.append((rp, A.col))
    for rp_np, col_np in cases:
        st = _noalloc(gnp, A.n, A.nnz, _dev(rp_np, torch.int32), _dev(col_np, torch.int32), val, out)
        assert st == 0, gnp.lib().gnp_last_error()
        torch.cuda.synchronize()
        assert np.isnan(out.item())
    # a well-formed call after the malformed ones clears the error flag
    st = _noalloc(gnp, A.n, A.nnz, _dev(A.row_ptr, torch.int32), _dev(A.col, torch.int32), val, out)
    assert st == 0
    torch.cuda.synchronize()
    assert out.item() == 8.0  # 5-point Poisson: gamma = 4 + 4 * 1
