"""CPU-side checks of the C-ABI boundary: the library builds for sm_103a,
loads, exports every entry point include/*.h declares, and rejects bad
arguments synchronously (no kernel is launched on these paths)."""
import ctypes
import subprocess

import pytest

import paper_0901_0638_gb300 as qm


def _read_text(path):
    with open(path) as fh:
        return fh.read()


@pytest.fixture(scope="module")
def lib():
    return qm.load()


def test_exports_every_declared_symbol(lib):
    names = qm.declared_symbols()
    assert "qm_normal_quantile_f32" in names and "qm_recycle" in names
    out = subprocess.run(["nm", "-D", "--defined-only", qm.LIB_PATH], capture_output=True,
                         text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if line.strip()}
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        getattr(lib, n)


def test_argument_errors_are_synchronous(lib):
    vp = ctypes.c_void_p
    assert lib.qm_normal_quantile_f32(None, None, 0, 0, None) == qm.QM_OK
    assert lib.qm_normal_quantile_f32(None, vp(4096), 8, 0, None) == qm.QM_ERR_INVALID
    assert "null" in qm.qm_last_error()
    # partial overlap of in and out
    assert lib.qm_normal_quantile_f64(vp(4096), vp(4096 + 8), 8, 0, None) == qm.QM_ERR_INVALID
    assert "overlap" in qm.qm_last_error()
    # a variant that does not exist in FP32
    assert lib.qm_normal_quantile_f32(vp(4096), vp(8192), 4, qm.QM_VAR_HYBRID_VOTE, None) == qm.QM_ERR_INVALID
    assert lib.qm_sample_fused(qm.QM_DIST_NORMAL, None, 1, 3, vp(4096), 0, 8, None, None) == qm.QM_ERR_INVALID
    assert lib.qm_sample_fused(qm.QM_DIST_NORMAL, None, 1, 0, None, 0, 8, None, None) == qm.QM_ERR_INVALID
    assert lib.qm_recycle(qm.QM_DIST_UNIFORM, qm.QM_DIST_EXPONENTIAL, None, vp(4096), vp(8192), 8,
                          None) == qm.QM_ERR_UNSUPPORTED
    assert lib.qm_philox_fill_u32(1, 0, None, 8, None) == qm.QM_ERR_INVALID


def test_batch_validation_before_any_launch(lib):
    vp = ctypes.c_void_p
    h = ctypes.c_void_p()
    seg = qm.qm_segment
    # unsupported pair
    arr = (seg * 1)(seg(qm.QM_DIST_UNIFORM, qm.QM_DIST_EXPONENTIAL, 0.0, 4096, 8192, 8))
    assert lib.qm_batch_create(arr, 1, None, ctypes.byref(h)) == qm.QM_ERR_INVALID
    # nu outside the supported range / invalid
    arr = (seg * 1)(seg(qm.QM_DIST_NORMAL, qm.QM_DIST_STUDENT_T, 150.0, 4096, 8192, 8))
    assert lib.qm_batch_create(arr, 1, None, ctypes.byref(h)) == qm.QM_ERR_UNSUPPORTED
    arr = (seg * 1)(seg(qm.QM_DIST_NORMAL, qm.QM_DIST_STUDENT_T, -2.0, 4096, 8192, 8))
    assert lib.qm_batch_create(arr, 1, None, ctypes.byref(h)) == qm.QM_ERR_INVALID
    # overlapping outputs of two segments
    arr = (seg * 2)(seg(qm.QM_DIST_EXPONENTIAL, qm.QM_DIST_NORMAL, 0.0, 4096, 1 << 20, 64),
                    seg(qm.QM_DIST_EXPONENTIAL, qm.QM_DIST_NORMAL, 0.0, 8192, (1 << 20) + 256, 64))
    assert lib.qm_batch_create(arr, 2, None, ctypes.byref(h)) == qm.QM_ERR_INVALID
    assert "overlap" in qm.qm_last_error()
    # null data pointer, bad tuning, empty table
    arr = (seg * 1)(seg(qm.QM_DIST_EXPONENTIAL, qm.QM_DIST_NORMAL, 0.0, None, 8192, 8))
    assert lib.qm_batch_create(arr, 1, None, ctypes.byref(h)) == qm.QM_ERR_INVALID
    arr = (seg * 1)(seg(qm.QM_DIST_EXPONENTIAL, qm.QM_DIST_NORMAL, 0.0, 4096, 8192, 8))
    assert lib.qm_batch_create(arr, 1, ctypes.byref(qm.qm_tuning(300, 2, 0)), ctypes.byref(h)) == qm.QM_ERR_INVALID
    assert lib.qm_batch_create(arr, 0, None, ctypes.byref(h)) == qm.QM_ERR_INVALID


def test_copula_validation_before_any_device_call(lib):
    import numpy as np
    L = np.ascontiguousarray(np.triu(np.ones((3, 3))))
    m = (qm.qm_margin * 3)(*[qm.qm_margin(qm.QM_DIST_NORMAL, 0.0)] * 3)
    h = ctypes.c_void_p()
    assert lib.qm_copula_create(3, L.ctypes.data, m, ctypes.byref(h)) == qm.QM_ERR_INVALID
    assert lib.qm_copula_create(17, L.ctypes.data, m, ctypes.byref(h)) == qm.QM_ERR_INVALID
    L = np.ascontiguousarray(np.eye(3))
    L[1, 1] = 0.0
    assert lib.qm_copula_create(3, L.ctypes.data, m, ctypes.byref(h)) == qm.QM_ERR_INVALID
    assert lib.qm_copula_sample(None, 1, 0, None, 8, None) == qm.QM_ERR_INVALID


def test_binding_constants_match_the_header():
    """Every numeric #define and enum value of include/qm.h that the binding
    also defines has the same value there (layouts and limits the tests and
    callers size buffers from)."""
    import os
    import re
    hdr = _read_text(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "qm.h"))
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    values = {}
    for name, expr in re.findall(r"^#define (QM_[A-Z0-9_]+) (.+)$", hdr, flags=re.M):
        try:
            values[name] = eval(expr, {}, dict(values))
        except Exception:
            pass
    for name, val in re.findall(r"\b(QM_[A-Z0-9_]+)\s*=\s*(-?\d+)\s*[,}\n]", hdr):
        values[name] = int(val)
    checked = 0
    for name, val in values.items():
        if hasattr(qm, name):
            assert getattr(qm, name) == val, (name, getattr(qm, name), val)
            checked += 1
    assert checked >= 20, checked
