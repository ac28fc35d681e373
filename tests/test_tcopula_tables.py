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
    j = np.clip(np.trunc(z * qm.QM_TC_HZ_INV + qm.QM_TC_Z_MAX * qm.QM_TC_HZ_INV).astype(int), 0, qm.QM_TC_NZ - 1)
    row = chi[j]
    s = z - row[:, 10]
    acc = row[:, 9].copy()
    for k in range(8, -1, -1):
        acc = acc * s + row[:, k]
    return acc


def eval_g(g, t):
    """The device's evaluation: exponent and top mantissa bits select the row
    (row 0 below 2^QM_TC_G_EMIN), r = m / m_c - 1 with 1/m_c from the row."""
    ne = (g.shape[0] - 1) >> qm.QM_TC_G_K
    a = np.abs(t)
    m, E = np.frexp(a)                           # a = m 2^E, m in [0.5, 1)
    E = np.where(a == 0, -1075, E - 1)
    m = m * 2.0                                  # m in [1, 2)
    small = E < qm.QM_TC_G_EMIN
    e = np.minimum(E - qm.QM_TC_G_EMIN, ne - 1)
    j = np.floor((m - 1.0) * (1 << qm.QM_TC_G_K)).astype(int)
    row = np.where(small, 0, 1 + (e << qm.QM_TC_G_K) + j)
    rp = g[row]
    v = np.where(small, a, m * rp[:, 10] - 1.0)
    acc = rp[:, 9].copy()
    for k in range(8, -1, -1):
        acc = acc * v + rp[:, k]
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
    ne = (g.shape[0] - 1) >> qm.QM_TC_G_K
    tmax = 2.0 ** (qm.QM_TC_G_EMIN + ne)
    # the largest |T| of the sampler: 8.3 * 4 * sqrt(nu / W(-8.3)) (< tmax)
    smax = math.sqrt(nu / oracle.chi2_from_normal(nu, np.array([-8.3]))[0])
    assert 33.2 * smax < tmax
    rng = np.random.default_rng(int(nu * 10))
    t = np.concatenate([rng.uniform(0, 2, 2000), np.exp(rng.uniform(math.log(1e-3), math.log(33.2 * smax), 3000)),
                        np.linspace(0, 2.2, 300), [1e-12, 1e-6, 2.0**-5, 2.0**-5 * (1 - 2**-52), 2.0, 33.2 * smax],
                        2.0 ** np.arange(-5, int(math.log2(33.2 * smax)))])
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
