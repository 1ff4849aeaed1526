"""The C-ABI library builds (nvcc cross-compiles sm_103a), loads without a
GPU, exports every function include/nfhmm.h declares, and rejects bad
arguments on the host before touching the device."""
import ctypes

import pytest


@pytest.fixture(scope="module")
def lib():
    from paper_1206_6468_gb300 import build
    build.build()
    from paper_1206_6468_gb300 import nfhmm
    return nfhmm


def test_exports_every_declared_function(lib):
    names = lib.declared_functions()
    assert len(names) >= 16
    missing = [n for n in names if not hasattr(lib._lib, n)]
    assert not missing, missing


def test_null_arguments_rejected(lib):
    init = lib.call_raw("nfhmm_vi_init")
    h = ctypes.c_void_p()
    d = lib.Dims(2, 4, 5, 129, 200, 1.0, 0, 0)
    assert init(ctypes.byref(h), ctypes.byref(d), None, None, None, None, 0, None) == lib.EINVAL
    assert h.value is None
    assert "NULL" in lib._lib.nfhmm_last_error().decode()
    assert lib.call_raw("nfhmm_vi_sweep")(None, 1, None) == lib.EINVAL
    out = ctypes.c_double()
    assert lib.call_raw("nfhmm_bound")(None, ctypes.byref(out)) == lib.EINVAL
    assert lib.call_raw("nfhmm_separate")(None, None, 1, 0, 0) == lib.EINVAL
    assert lib.call_raw("nfhmm_get_posteriors")(None, None, 0) == lib.EINVAL
    assert lib.call_raw("nfhmm_forward_backward")(1, 2, 3, None, None, None, None, None, 0,
                                                  None) == lib.EINVAL
    assert lib.call_raw("nfhmm_kernel_launches")(None) == 0
    lib.call_raw("nfhmm_destroy")(None)


@pytest.mark.parametrize("dims,msg", [
    ((0, 4, 5, 129, 200, 1.0, 0, 0), ">= 1"),
    ((2, 4, 5, 129, 0, 1.0, 0, 0), ">= 1"),
    ((2, 65, 5, 129, 200, 1.0, 0, 0), "N must be"),
    ((2, 4, 5, 129, 200, -1.0, 0, 0), "gamma"),
    ((2, 4, 5, 129, 200, 1.0, 7, 0), "precision"),
    ((2, 4, 5, 129, 200, 1.0, 0, 9), "init_mode"),
])
def test_bad_dims_rejected(lib, dims, msg):
    import numpy as np
    buf = np.zeros(16, dtype=np.float32)
    p = ctypes.c_void_p(buf.ctypes.data)
    h = ctypes.c_void_p()
    d = lib.Dims(*dims)
    rc = lib.call_raw("nfhmm_vi_init")(ctypes.byref(h), ctypes.byref(d), p, p, p, p, 0, None)
    assert rc == lib.EINVAL
    assert msg in lib._lib.nfhmm_last_error().decode()
