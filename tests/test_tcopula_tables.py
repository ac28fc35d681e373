"""The t-copula recycling tables (Sec. 9), on the CPU.

qm_tcopula_table_build returns, for one nu, the two host-built tables the
t-copula sampler reads: log W(z) for the chi-squared mixing variable and
G(t) = Phi^{-1}(F_nu(t)) for the margins.  Evaluated here in numpy in the
device's order, they must match the oracle (pinned in test_tcopula_oracle.py)
to 1e-12 relative over the whole range the sampler uses: every 53-bit grid
normal for W, and |T| up to the largest value the sampler can produce for G.
"""
import math

import numpy as np
import pytest

import oracle
import paper_0901_0638_gb300 as qm

NUS = [0.75, 1.0, 2.0, 3.3, 4.0, 30.0, 100.0]


def eval_log_w(chi, z):
    j = np.clip(np.floor((z + qm.QM_TC_Z_MAX) * qm.QM_TC_HZ_INV).astype(int), 0, qm.QM_TC_NZ - 1)
    s = z - (-qm.QM_TC_Z_MAX + (j + 0.5) / qm.QM_TC_HZ_INV)
    c = chi[j]
    acc = c[:, 9].copy()
    for k in range(8, -1, -1):
        acc = acc * s + c[:, k]
    return acc


def eval_g(g, t):
    nb = g.shape[0] - qm.QM_TC_NA
    a = np.abs(t)
    small = a < 2.0
    row = np.empty(a.shape, dtype=int)
    s = np.empty_like(a)
    j = np.minimum((a[small] * qm.QM_TC_HT_INV).astype(int), qm.QM_TC_NA - 1)
    row[small] = j
    s[small] = a[small] - np.where(j == 0, 0.0, (j + 0.5) / qm.QM_TC_HT_INV)
    y = np.log(a[~small])
    i = np.clip(((y - math.log(2)) * qm.QM_TC_HT_INV).astype(int), 0, nb - 1)
    row[~small] = qm.QM_TC_NA + i
    s[~small] = y - (math.log(2) + (i + 0.5) / qm.QM_TC_HT_INV)
    c = g[row]
    acc = c[:, 9].copy()
    for k in range(8, -1, -1):
        acc = acc * s + c[:, k]
    return np.copysign(acc, t)


@pytest.mark.parametrize("nu", NUS)
def test_mixing_table_against_the_oracle(nu):
    chi, _ = qm.qm_tcopula_table_build(nu)
    rng = np.random.default_rng(int(nu * 100))
    z = np.concatenate([rng.uniform(-8.3, 8.3, 3000), np.linspace(-8.2924, 8.2924, 533), [0.0, -1e-9]])
    w = np.exp(eval_log_w(chi, z))
    ref = oracle.chi2_from_normal(nu, z)
    r = np.abs(w / ref - 1)
    assert r.max() < 1e-12, (z[np.argmax(r)], r.max())


@pytest.mark.parametrize("nu", NUS)
def test_t_to_normal_table_against_the_oracle(nu):
    chi, g = qm.qm_tcopula_table_build(nu)
    nb = g.shape[0] - qm.QM_TC_NA
    tmax = math.exp(math.log(2) + nb / qm.QM_TC_HT_INV)
    # the largest |T| of the sampler: 8.3 * 4 * sqrt(nu / W(-8.3)) (< tmax)
    smax = math.sqrt(nu / oracle.chi2_from_normal(nu, np.array([-8.3]))[0])
    assert 33.2 * smax < tmax
    rng = np.random.default_rng(int(nu * 10))
    t = np.concatenate([rng.uniform(0, 2, 2000), np.exp(rng.uniform(math.log(2), math.log(33.2 * smax), 3000)),
                        np.linspace(0, 2.2, 300), [1e-12, 1e-6, 2.0, 33.2 * smax]])
    t = np.concatenate([t, -t[::7]])
    got = eval_g(g, t)
    ref = oracle.t_to_normal(nu, t)
    nz = ref != 0
    r = np.abs(got[nz] / ref[nz] - 1)
    assert r.max() < 1e-12, (t[nz][np.argmax(r)], r.max())
    assert np.all(got[~nz] == 0)


def test_unsupported_nu():
    for nu in (0.5, 150.0):
        with pytest.raises(qm.QMError) as e:
            qm.qm_tcopula_table_build(nu)
        assert e.value.status == qm.QM_ERR_UNSUPPORTED
