"""The C-ABI library loads, exports every symbol its header declares, and
rejects bad arguments before touching CUDA (CPU only: no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "qs.h")


@pytest.fixture(scope="module")
def qs():
    from paper_2506_09198_gb300 import build

    build.build()
    from paper_2506_09198_gb300 import qs as mod

    return mod


def declared_functions():
    text = open(HEADER).read()
    return sorted(set(re.findall(r"^\s*(?:qs_status|const char\*)\s+(qs_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("qs_create", "qs_apply_1q", "qs_apply_2q", "qs_apply_ctrl", "qs_apply_diag",
                     "qs_apply_perm", "qs_fuse_run", "qs_batch_run", "qs_norm", "qs_probs", "qs_sync"):
        assert required in names


def test_every_declared_symbol_is_exported(qs):
    lib = qs.lib()
    for name in declared_functions():
        assert hasattr(lib, name), f"{name} declared in qs.h but not exported"
    assert sorted(qs.EXPORTED) == declared_functions()


def test_argument_validation_without_gpu(qs):
    lib = qs.lib()
    h = ctypes.c_void_p()
    assert lib.qs_create(0, qs.QS_C128, ctypes.byref(h)) == qs.QS_ERR_ARG
    assert "n = 0" in qs.qs_last_error()
    assert lib.qs_create(35, qs.QS_C128, ctypes.byref(h)) == qs.QS_ERR_ARG
    assert lib.qs_create(36, qs.QS_C64, ctypes.byref(h)) == qs.QS_ERR_ARG
    assert lib.qs_create(10, 7, ctypes.byref(h)) == qs.QS_ERR_ARG
    assert lib.qs_create(10, qs.QS_C64, None) == qs.QS_ERR_ARG
    U = (ctypes.c_double * 8)()
    assert lib.qs_apply_1q(None, 0, U) == qs.QS_ERR_ARG
    assert lib.qs_norm(None, None) == qs.QS_ERR_ARG
    assert lib.qs_sync(None, 1.0) == qs.QS_ERR_ARG
    assert lib.qs_destroy(None) == qs.QS_OK
    assert lib.qs_wrap(10, qs.QS_C128, None, None, ctypes.byref(h)) == qs.QS_ERR_ARG
    assert lib.qs_batch_run(None, None, -1, None) == qs.QS_ERR_ARG
    b = ctypes.c_void_p()
    assert lib.qs_batch_compile(None, None, 0, ctypes.byref(b)) == qs.QS_ERR_ARG
    assert lib.qs_batch_compile(None, None, 1, None) == qs.QS_ERR_ARG
    assert lib.qs_batch_launch(None) == qs.QS_ERR_ARG
    assert lib.qs_batch_destroy(None) == qs.QS_OK
    for bad in (-1.0, 61.0, float("nan")):
        assert lib.qs_set_wait_limit(bad) == qs.QS_ERR_ARG
    assert lib.qs_set_wait_limit(2.0) == qs.QS_OK
    t3 = (ctypes.c_int * 3)(0, 1, 2)
    U8 = (ctypes.c_double * 128)()
    assert lib.qs_apply_dense(None, None, 0, t3, 3, U8) == qs.QS_ERR_ARG
    assert lib.qs_set_tensor_cores(None, 1) == qs.QS_ERR_ARG
    for args in ((12, qs.QS_C128, 0, 1), (12, qs.QS_C128, 7, 1), (11, qs.QS_C128, 2, 1), (13, qs.QS_C128, 2, 5),
                 (12, 9, 1, 1)):
        assert lib.qs_create_split(*args, ctypes.byref(h)) == qs.QS_ERR_ARG
    assert lib.qs_create_split(12, qs.QS_C128, 1, 1, None) == qs.QS_ERR_ARG
    assert qs.qs_version().startswith("libqs")


def test_noalloc_rejects_host_memory_without_gpu(qs):
    """A host buffer is never handed to a kernel: without a GPU the call fails
    at the device lookup, with a GPU at the pointer check (QS_ERR_ARG)."""
    import numpy as np

    lib = qs.lib()
    host = np.zeros(1 << 10, dtype=np.complex128)
    out = np.zeros(4, dtype=np.float64)
    q = (ctypes.c_int * 2)(0, 1)
    st = lib.qs_probs_noalloc(ctypes.c_void_p(host.ctypes.data), 10, qs.QS_C128, q, 2,
                              ctypes.c_void_p(out.ctypes.data), None)
    assert st != qs.QS_OK
    assert np.all(out == 0.0)


def test_binding_raises_qserror(qs):
    with pytest.raises(qs.QSError) as e:
        qs.qs_create(0, qs.QS_C64)
    assert e.value.status == qs.QS_ERR_ARG
