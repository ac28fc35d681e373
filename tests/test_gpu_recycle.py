"""GPU parity of the recycling maps against the CPU FP64 oracle.

Normal -> Student t, Q_nu(z) = F_nu^{-1}(Phi(z)) (Sec. 3), for every
tabulated nu and for untabulated real nu (tables built on the host at first
use); tolerance 1e-12 relative (exact for 0, infinities and NaN)."""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_0901_0638_gb300 as qm
from paper_0901_0638_gb300 import workloads as W
from tests.gpu_util import f64_violations, rel_err

pytestmark = pytest.mark.gpu
DEV = "cuda"
NUS = [1.0, 2.0, 3.0, 4.0, 5.0, 8.0, 10.0, 30.0]


def run_t(nu, z):
    t = torch.from_numpy(np.ascontiguousarray(z, dtype=np.float64)).to(DEV)
    out = torch.empty_like(t)
    qm.qm_recycle(qm.QM_DIST_NORMAL, qm.QM_DIST_STUDENT_T, t, out, nu=nu)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def z_cases():
    segs = np.arange(0, 281) / 32.0
    return np.concatenate([
        W.normal_box_muller(4, 1 << 17).numpy(),
        np.linspace(-12, 12, 4801),
        segs, np.nextafter(segs, 0), np.nextafter(segs, 20),            # segment edges
        [8.75, np.nextafter(8.75, 0), 9.0, 15.0, 25.0, 37.0, 1e-300, 1e-12, -1e-12, 0.0, -0.0,
         np.inf, -np.inf, np.nan],
    ])


@pytest.mark.parametrize("nu", NUS)
def test_recycle_normal_to_t(nu):
    z = z_cases()
    w = oracle.recycle_t(nu, z)
    t = run_t(nu, z)
    r = rel_err(t, w)
    print(f"nu={nu}: max rel {r.max():.3g}")
    assert not f64_violations(t, w, 1e-12).any()
    # exact oddness, including signed zeros
    assert np.array_equal(run_t(nu, -z[np.isfinite(z)]), -t[np.isfinite(z)])
    assert math.copysign(1.0, t[-4]) == -1.0


@pytest.mark.parametrize("nu", [0.75, 1.5, 2.5, 6.3, 17.0, 50.0, 100.0])
def test_recycle_normal_to_t_any_nu(nu):
    z = z_cases()
    w = oracle.recycle_t(nu, z)
    t = run_t(nu, z)
    r = rel_err(t, w)
    print(f"nu={nu} (run-time table): max rel {r.max():.3g}")
    assert not f64_violations(t, w, 1e-12).any()
    assert np.array_equal(run_t(nu, -z[np.isfinite(z)]), -t[np.isfinite(z)])
    assert np.array_equal(run_t(nu, z), t, equal_nan=True)   # second call: cached table, same result


def test_recycle_t_argument_errors():
    z = torch.zeros(4, dtype=torch.float64, device=DEV)
    for nu in (0.5, 150.0):
        with pytest.raises(qm.QMError) as e:
            qm.qm_recycle(qm.QM_DIST_NORMAL, qm.QM_DIST_STUDENT_T, z, z, nu=nu)
        assert e.value.status == qm.QM_ERR_UNSUPPORTED
    with pytest.raises(qm.QMError) as e:
        qm.qm_recycle(qm.QM_DIST_NORMAL, qm.QM_DIST_STUDENT_T, z, z, nu=-1.0)
    assert e.value.status == qm.QM_ERR_INVALID


@pytest.mark.parametrize("nu", [1.0, 4.0, 30.0, 6.5])
def test_fused_student_t(nu):
    n = (1 << 15) + 3
    key, ctr0 = 21, 0
    words = oracle.philox_stream(key, ctr0, 2 * n + 2).astype(np.uint64)
    kk = (((words[0::2] >> 11) << 32) | words[1::2])[:n]
    upper = kk >= 2**52
    d = (np.where(upper, 2**53 - 1 - kk, kk).astype(np.float64) + 0.5) * 2.0**-53
    zn = oracle.probit(d)
    zn = np.where(upper, -zn, zn)
    w = oracle.recycle_t(nu, zn)
    out = torch.empty(n, dtype=torch.float64, device=DEV)
    qm.qm_sample_fused(qm.QM_DIST_STUDENT_T, key, ctr0, out, out_is_f64=True, nu=nu)
    torch.cuda.synchronize()
    assert not f64_violations(out.cpu().numpy(), w, 1e-12).any()
