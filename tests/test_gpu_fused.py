"""GPU parity of the Philox stream, the fused generate+transform path and the
exponential -> normal recycling map."""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_0901_0638_gb300 as qm
from paper_0901_0638_gb300 import workloads as W
from tests.gpu_util import f32_violations, f64_violations, rel_err

pytestmark = pytest.mark.gpu
DEV = "cuda"


@pytest.mark.parametrize("key,ctr0,n", [(1, 0, 10001), (3, 3, 4097), (2**40 + 7, 4 * (2**32 - 1) - 2, 1000)])
def test_philox_fill_matches_oracle(key, ctr0, n):
    out = torch.empty(n, dtype=torch.int32, device=DEV)
    qm.qm_philox_fill_u32(key, ctr0, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint32)
    assert np.array_equal(got, oracle.philox_stream(key, ctr0, n))


@pytest.mark.parametrize("n", [(1 << 20) + 3, 17, 4])
def test_fused_equals_unfused_bit_exact(n):
    key, ctr0 = 3, 4 * 1000
    fused = torch.empty(n, dtype=torch.float32, device=DEV)
    qm.qm_sample_fused(qm.QM_DIST_NORMAL, key, ctr0, fused)
    words = torch.empty(n, dtype=torch.int32, device=DEV)
    qm.qm_philox_fill_u32(key, ctr0, words)
    unfused = torch.empty(n, dtype=torch.float32, device=DEV)
    qm.qm_normal_quantile_bits24_f32(words, unfused)
    torch.cuda.synchronize()
    assert torch.equal(fused, unfused)
    # and against the oracle on the exact grid point
    k = oracle.philox_stream(key, ctr0, n) >> 8
    w = oracle.probit((k.astype(np.float64) + 0.5) * 2.0**-24)
    assert not f32_violations(fused.cpu().numpy(), w).any()


def test_fused_moments_against_fp64_reduction_and_normal_law():
    n = 1 << 24
    out = torch.empty(n, dtype=torch.float32, device=DEV)
    mom = torch.empty(4, dtype=torch.float64, device=DEV)
    qm.qm_sample_fused(qm.QM_DIST_NORMAL, 3, 0, out, moments4=mom)
    mom_only = torch.empty(4, dtype=torch.float64, device=DEV)
    qm.qm_sample_fused(qm.QM_DIST_NORMAL, 3, 0, None, n=n, moments4=mom_only)
    torch.cuda.synchronize()
    assert torch.equal(mom, mom_only)                 # fixed reduction order
    z = out.double()
    ref = torch.stack([z.sum(), (z**2).sum(), (z**3).sum(), (z**4).sum()])
    absz = z.abs()
    scale = torch.stack([absz.sum(), (absz**2).sum(), (absz**3).sum(), (absz**4).sum()])
    # FP32 partials over 64 samples: per-sample rounding <= ~(64 + 3) 2^-24
    # of |z|^k, so the sums agree to that fraction of sum |z|^k.
    assert torch.all((mom - ref).abs() <= 67 * 2.0**-24 * scale), (mom, ref)
    m = (mom / n).cpu().numpy()
    # 5 sigma bounds for the sample moments of N(0,1) at n = 2^24
    sd = np.sqrt(np.array([1.0, 2.0, 15.0, 96.0]) / n)
    assert np.all(np.abs(m - np.array([0.0, 1.0, 0.0, 3.0])) <= 5 * sd), m


def test_fused_f64_normal_and_exponential():
    n = (1 << 16) + 1
    key, ctr0 = 11, 8
    words = oracle.philox_stream(key, ctr0, 2 * n + 2).astype(np.uint64)
    kk = ((words[0::2] >> 11) << 32) | words[1::2]
    kk = kk[:n]
    upper = kk >= 2**52
    j = np.where(upper, 2**53 - 1 - kk, kk).astype(np.float64)
    d = (j + 0.5) * 2.0**-53
    u_lo = d                                              # exact
    out = torch.empty(n, dtype=torch.float64, device=DEV)
    qm.qm_sample_fused(qm.QM_DIST_NORMAL, key, ctr0, out, out_is_f64=True)
    torch.cuda.synchronize()
    w = oracle.probit(u_lo)
    w = np.where(upper, -w, w)
    assert not f64_violations(out.cpu().numpy(), w, 4e-15).any()
    # exponential samples x = -log(u) mapped to the normal
    qm.qm_sample_fused(qm.QM_DIST_EXPONENTIAL, key, ctr0, out, out_is_f64=True)
    torch.cuda.synchronize()
    x = np.where(upper, -np.log1p(-d), -np.log(d))
    w = oracle.recycle_exp(x)
    z = out.cpu().numpy()
    # x is formed on the device with its own log/log1p (within an ulp or so of
    # numpy's); the map's slope dz/dx = e^{-x}/phi(z) turns that into an
    # absolute difference, which dominates where z is near 0 (x near ln 2).
    slope = np.exp(-x) / (np.exp(-0.5 * w * w) / np.sqrt(2 * np.pi))
    tol = 1e-12 * np.abs(w) + 4 * 2.2e-16 * x * slope
    assert np.all(np.abs(z - w) <= tol)


def test_recycle_exp_to_normal():
    x = np.concatenate([
        W.exponential(4, 1 << 20).numpy(),
        10.0 ** -np.linspace(0, 300, 301), np.linspace(0.01, 40, 4001), np.linspace(40, 744, 300),
        math.log(2) + np.arange(-40, 41) * 2.0**-53,
        [0.0, np.inf, -1.0, np.nan, 0.28768207245178093, 1.3862943611198906, 0.35],
        # segment and region boundaries of the evaluation: v = x - ln 2 at
        # j/32 and q/8 (segment ends), v = -1/64 (the central piece), the
        # binade and segment starts of x below ln 2, x = 2^-26, v = 64
        np.array([math.log(2) + j / 32 + dd for j in range(1, 32) for dd in (-1e-16, 0.0, 1e-16)]),
        np.array([math.log(2) + q / 8 + dd for q in range(8, 512, 7) for dd in (-1e-15, 0.0, 1e-15)]),
        math.log(2) - 1 / 64 + np.array([-1e-17, 0.0, 2e-17, 1e-16]),
        np.array([np.nextafter(2.0**E * (1 + j / 32), to) for E in range(-26, 0) for j in (0, 1, 15, 31)
                  for to in (0.0, 1.0)]),
        [2.0**-26, np.nextafter(2.0**-26, 0.0), np.nextafter(2.0**-26, 1.0), math.log(2) + 64.0,
         np.nextafter(math.log(2) + 64.0, 0.0)],
        # the device rows: 64 segments in every binade of x from 2^-26 to 128,
        # the segment [0.6875, 0.6953125) that holds ln 2 and its neighbours
        np.array([np.nextafter(2.0**E * (1 + j / 64), to) for E in range(-26, 7) for j in (0, 1, 23, 24, 25, 63)
                  for to in (0.0, 2.0**E * (1 + j / 64), 1e9)]),
        # where the centre row hands over: |x - ln 2| = 2^-12
        np.array([math.log(2) + sg * 2.0**-12 * f for sg in (-1.0, 1.0) for f in (1 - 1e-12, 1.0, 1 + 1e-12)]),
    ])
    w = oracle.recycle_exp(x)
    t = torch.from_numpy(x).to(DEV)
    z = torch.empty_like(t)
    qm.qm_recycle(qm.QM_DIST_EXPONENTIAL, qm.QM_DIST_NORMAL, t, z)
    torch.cuda.synchronize()
    z = z.cpu().numpy()
    r = rel_err(z, w)
    print(f"exp->normal max rel {r.max():.3g}")
    assert not f64_violations(z, w, 1e-12).any()
