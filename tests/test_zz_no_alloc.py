"""The allocation-free moments entry point (qm_sample_moments_noalloc).

Callers that cannot allocate at call time -- a latency-bound pipeline that
cannot let cudaMalloc synchronise the device, an embedded runtime that plans
all device memory up front, code that runs while a caching allocator holds its
lock -- get the fused Philox -> normal moments from a static scratch array.
This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test.  It must pass alone in a fresh
process and after the other tests.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_0901_0638_gb300 as qm

pytestmark = pytest.mark.gpu


def _sums_reference(n, key, ctr0):
    mom = torch.empty(4, dtype=torch.float64, device="cuda")
    qm.qm_sample_fused(qm.QM_DIST_NORMAL, key, ctr0, None, n=n, moments4=mom)
    out = torch.empty(n, dtype=torch.float32, device="cuda")
    qm.qm_sample_fused(qm.QM_DIST_NORMAL, key, ctr0, out)
    z = out.double().abs()
    scale = torch.stack([z.sum(), (z ** 2).sum(), (z ** 3).sum(), (z ** 4).sum()])
    return mom, scale


def test_noalloc_matches_allocating_path_twice_in_a_row():
    lib = qm.load()
    stream = torch.cuda.current_stream().cuda_stream
    for n, key, ctr0 in [((1 << 22) + 5, 3, 0), (1 << 20, 9, 400)]:
        ref, scale = _sums_reference(n, key, ctr0)
        got = []
        for _ in range(2):                       # two calls in a row share the scratch
            m = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
            st = lib.qm_sample_moments_noalloc(ctypes.c_uint64(key), ctypes.c_uint64(ctr0),
                                               ctypes.c_size_t(n), ctypes.c_void_p(m.data_ptr()),
                                               ctypes.c_void_p(stream))
            assert st == qm.QM_OK, qm.qm_last_error()
            got.append(m)
        torch.cuda.synchronize()
        # same samples; both sum FP32 partials over 64 samples in FP64, each
        # within (64 + 3) 2^-24 of sum |z|^k, so they agree to twice that
        for m in got:
            assert torch.all((m - ref).abs() <= 2 * 67 * 2.0 ** -24 * scale), (m, ref)
        assert torch.equal(got[0], got[1])


def test_noalloc_moments_against_oracle_samples():
    """Independently of the library's other paths: the same samples from
    the oracle (its own Philox stream and FP64 quantile at the exact grid
    points (k + 1/2) 2^-24), summed in FP64.  Each device sample is within
    4 ulp (2^-21 relative) of the exact value, so its k-th power within
    k 2^-21, plus the FP32 partial sums' (64 + 3) 2^-24."""
    lib = qm.load()
    n, key, ctr0 = (1 << 18) + 5, 3, 64
    k = oracle.philox_stream(key, ctr0, n) >> 8
    z = oracle.probit((k.astype(np.float64) + 0.5) * 2.0 ** -24)
    ref = np.array([np.sum(z ** p) for p in (1, 2, 3, 4)])
    scale = np.array([np.sum(np.abs(z) ** p) for p in (1, 2, 3, 4)])
    m = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    st = lib.qm_sample_moments_noalloc(ctypes.c_uint64(key), ctypes.c_uint64(ctr0), ctypes.c_size_t(n),
                                       ctypes.c_void_p(m.data_ptr()), ctypes.c_void_p(None))
    assert st == qm.QM_OK, qm.qm_last_error()
    torch.cuda.synchronize()
    got = m.cpu().numpy()
    tol = (67 * 2.0 ** -24 + np.array([1, 2, 3, 4]) * 2.0 ** -21) * scale
    assert np.all(np.abs(got - ref) <= tol), (got, ref)


def test_noalloc_rejects_oversize_and_bad_arguments():
    lib = qm.load()
    m = torch.empty(4, dtype=torch.float64, device="cuda")
    st = lib.qm_sample_moments_noalloc(ctypes.c_uint64(1), ctypes.c_uint64(0),
                                       ctypes.c_size_t((1 << 32) + 1), ctypes.c_void_p(m.data_ptr()),
                                       ctypes.c_void_p(None))
    assert st == qm.QM_ERR_INVALID and "static scratch limit" in qm.qm_last_error()
    st = lib.qm_sample_moments_noalloc(ctypes.c_uint64(1), ctypes.c_uint64(2),
                                       ctypes.c_size_t(16), ctypes.c_void_p(m.data_ptr()),
                                       ctypes.c_void_p(None))
    assert st == qm.QM_ERR_INVALID
