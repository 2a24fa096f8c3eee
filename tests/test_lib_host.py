"""CPU-only checks of the C-ABI library: it builds for sm_103a, loads without a GPU,
exports every function include/gnp.h declares, the binding declares each of them, and
the host-side logic (argument and CSR validation, weight counts, status names) works
without touching the device."""
import ctypes as C
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared_functions():
    names = []
    for h in HEADERS:
        txt = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_]\w*\s*\**\s+\**([A-Za-z_]\w*)\s*\(", txt, re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def lib():
    from paper_2406_00809_gb300 import build
    build.build()
    from paper_2406_00809_gb300 import gnp
    return gnp.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("gnp_mat_create", "gnp_create", "gnp_apply", "gnp_train_step", "fgmres_solve",
                 "gnp_get_weights", "gnp_destroy", "gnp_mat_destroy", "gnp_last_error"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_every_symbol():
    src = open(os.path.join(ROOT, "paper_2406_00809_gb300", "gnp.py")).read()
    missing = [n for n in declared_functions() if f'"{n}"' not in src]
    assert not missing, missing


def test_weight_count_and_status_strings(lib):
    assert lib.gnp_weight_count(8) == 5265  # 592 + 8*512 + 577
    assert lib.gnp_weight_count(0) == 1169
    assert lib.gnp_weight_count(-1) == -1
    assert lib.gnp_status_string(0) == b"GNP_OK"
    assert lib.gnp_status_string(7) == b"GNP_ERR_RESIDUAL_MISMATCH"


def _create(lib, rp, col, val, n=None):
    rp = np.ascontiguousarray(rp, dtype=np.int32)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.float64)
    out = C.c_void_p()
    n = rp.size - 1 if n is None else n
    return lib.gnp_mat_create(n, col.size, rp.ctypes.data, col.ctypes.data, val.ctypes.data, 0, None,
                              C.byref(out)), out


def test_csr_validation_happens_on_the_host(lib):
    # column out of range
    s, out = _create(lib, [0, 1, 2], [0, 2], [1.0, 1.0])
    assert s == 2 and not out.value
    assert b"col[1]" in lib.gnp_last_error()
    # decreasing row pointer
    s, _ = _create(lib, [0, 2, 1, 3], [0, 1, 2], [1.0, 1.0, 1.0])
    assert s == 2 and b"decreases" in lib.gnp_last_error()
    # row_ptr[n] != nnz
    s, _ = _create(lib, [0, 1, 3], [0, 1], [1.0, 1.0])
    assert s == 2
    # n < 1
    s, _ = _create(lib, [0], [], [], n=0)
    assert s == 1


def test_null_arguments_are_rejected(lib):
    assert lib.gnp_apply(None, None, None, None) == 1
    assert lib.fgmres_solve(None, None, None, None, 10, 1e-8, 100, None, None) == 1
    assert lib.gnp_create(None, None, None, C.byref(C.c_void_p())) == 1
    assert b"null" in lib.gnp_last_error()
