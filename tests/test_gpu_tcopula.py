"""t copula with recycled marginals (Sec. 9 folding) on the GPU.

* Element by element against a numpy reference built from the oracle at the
  same Philox draws: normal 0 of a sample through the oracle's chi-squared
  map (W), normals 1..d through L, T_j = y_j / sigma_j sqrt(nu / W), margins
  by the oracle's Student t -> normal map and normal -> t map.
* Distribution checks that do not use the tables: Kendall's tau of an
  elliptical copula is (2/pi) arcsin(rho); a margin of the copula's own nu is
  Student t with nu degrees of freedom, a normal margin is N(0, 1)
  (Kolmogorov-Smirnov at 2^18 samples).
"""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_0901_0638_gb300 as qm

pytestmark = pytest.mark.gpu
DEV = "cuda"


def grid_normals(key, ctr0, n, count):
    nb = (count + 1) // 2
    w = oracle.philox_stream(key, ctr0, 4 * nb * n).astype(np.uint64).reshape(n, nb, 4)
    m = np.stack([((w[..., 0] >> 11) << 32) | w[..., 1], ((w[..., 2] >> 11) << 32) | w[..., 3]], axis=-1)
    m = m.reshape(n, 2 * nb)[:, :count]
    upper = m >= 2**52
    dd = (np.where(upper, 2**53 - 1 - m, m).astype(np.float64) + 0.5) * 2.0**-53
    e = oracle.probit(dd.ravel()).reshape(dd.shape)
    return np.where(upper, -e, e)


def reference(L, margins, nu, key, ctr0, n):
    d = L.shape[0]
    e = grid_normals(key, ctr0, n, d + 1)
    W = oracle.chi2_from_normal(nu, e[:, 0])
    S = np.sqrt(nu / W)
    eps = e[:, 1:]
    sigma = np.sqrt((L * L).sum(axis=1))
    y = eps @ L.T
    T = y / sigma * S[:, None]
    x = np.empty_like(T)
    for j, (kind, mu) in enumerate(margins):
        if kind == qm.QM_DIST_STUDENT_T and mu == nu:
            x[:, j] = T[:, j]
        else:
            g = oracle.t_to_normal(nu, T[:, j])
            x[:, j] = oracle.recycle_t(mu, g) if kind == qm.QM_DIST_STUDENT_T else g
    scale = (np.abs(eps) @ np.abs(L).T) / sigma * S[:, None]          # rounding scale of T
    return x, T, scale


@pytest.mark.parametrize("nu", [4.0, 0.75, 2.7, 30.0])
def test_tcopula_against_reference(nu):
    rng = np.random.default_rng(int(10 * nu))
    d = 6
    A = rng.normal(size=(d, d))
    C = A @ A.T + d * np.eye(d)
    L = np.linalg.cholesky(C)                        # a covariance: the copula is its correlation's
    margins = [(qm.QM_DIST_STUDENT_T, nu), (qm.QM_DIST_NORMAL, 0.0), (qm.QM_DIST_STUDENT_T, 4.0),
               (qm.QM_DIST_STUDENT_T, 2.3), (qm.QM_DIST_NORMAL, 0.0), (qm.QM_DIST_STUDENT_T, nu)]
    c = qm.Copula(L, margins, nu=nu)
    n, key, ctr0 = 3001, 23, 16
    out = torch.empty(d * n, dtype=torch.float64, device=DEV)
    c.sample(key, ctr0, out, n)
    torch.cuda.synchronize()
    x = out.cpu().numpy().reshape(d, n).T
    w, T, scale = reference(L, margins, nu, key, ctr0, n)
    for j in range(d):
        gain = np.abs(w[:, j] / np.where(T[:, j] == 0, 1, T[:, j]))
        tol = 1e-12 * np.abs(w[:, j]) + 1e-15 * scale[:, j] * np.maximum(gain, 1.0)
        bad = np.abs(x[:, j] - w[:, j]) > tol
        assert not bad.any(), (j, int(bad.sum()), x[bad, j][:3], w[bad, j][:3])
    c.close()


def kendall_tau(a, b):
    from scipy import stats
    return stats.kendalltau(a, b).statistic


def test_tcopula_distribution():
    from scipy import stats
    nu = 3.0
    R = np.array([[1.0, 0.7, -0.3], [0.7, 1.0, 0.2], [-0.3, 0.2, 1.0]])
    L = np.linalg.cholesky(R)
    c = qm.Copula(L, [(qm.QM_DIST_STUDENT_T, nu), (qm.QM_DIST_NORMAL, 0.0), (qm.QM_DIST_STUDENT_T, 6.0)], nu=nu)
    n = 1 << 18
    out = torch.empty(3 * n, dtype=torch.float64, device=DEV)
    c.sample(31, 0, out, n)
    x = out.view(3, n).cpu().numpy()
    c.close()
    sub = slice(0, 1 << 16)
    for (i, j) in ((0, 1), (0, 2), (1, 2)):
        tau = kendall_tau(x[i, sub], x[j, sub])
        assert abs(tau - 2 / math.pi * math.asin(R[i, j])) < 0.02, (i, j, tau)
    assert stats.kstest(x[0], stats.t(nu).cdf).statistic < 1.95 / math.sqrt(n)
    assert stats.kstest(x[1], stats.norm.cdf).statistic < 1.95 / math.sqrt(n)
    assert stats.kstest(x[2], stats.t(6.0).cdf).statistic < 1.95 / math.sqrt(n)


def test_tcopula_argument_errors():
    with pytest.raises(qm.QMError) as e:
        qm.Copula(np.eye(2), [(qm.QM_DIST_NORMAL, 0.0)] * 2, nu=0.5)
    assert e.value.status == qm.QM_ERR_UNSUPPORTED
    with pytest.raises(qm.QMError) as e:
        qm.Copula(np.triu(np.ones((2, 2))), [(qm.QM_DIST_NORMAL, 0.0)] * 2, nu=4.0)
    assert e.value.status == qm.QM_ERR_INVALID
    with pytest.raises(qm.QMError) as e:
        qm.Copula(np.eye(2), [(qm.QM_DIST_EXPONENTIAL, 0.0)] * 2, nu=4.0)
    assert e.value.status == qm.QM_ERR_UNSUPPORTED


@pytest.mark.parametrize("d,n", [(1, 1), (1, 257), (16, 3), (16, 1025), (7, 130)])
def test_copulas_dimensions_and_ragged_counts(d, n):
    """The degenerate dimension 1 and the maximum 16, ragged sample counts,
    a nonzero counter base: both copulas element by element, and nothing
    written past the d n outputs."""
    rng = np.random.default_rng(d * 1000 + n)
    A = rng.normal(size=(d, d))
    L = np.linalg.cholesky(A @ A.T + d * np.eye(d))
    kinds = [(qm.QM_DIST_NORMAL, 0.0), (qm.QM_DIST_STUDENT_T, 3.0), (qm.QM_DIST_STUDENT_T, 5.5)]
    margins = [kinds[j % 3] for j in range(d)]
    key, ctr0 = 77, 4 * 12345
    for nu in (None, 3.0):
        c = qm.Copula(L, margins, nu=nu)
        out = torch.full((d * n + 8,), 7.0, dtype=torch.float64, device=DEV)
        c.sample(key, ctr0, out, n)
        torch.cuda.synchronize()
        c.close()
        o = out.cpu().numpy()
        assert np.all(o[d * n:] == 7.0)
        x = o[: d * n].reshape(d, n).T
        if nu is None:
            e = grid_normals(key, ctr0, n, d)
            sigma = np.sqrt((L * L).sum(axis=1))
            y = e @ L.T / sigma
            ref = np.stack([oracle.recycle_t(mu, y[:, j]) if k == qm.QM_DIST_STUDENT_T else y[:, j]
                            for j, (k, mu) in enumerate(margins)], axis=1)
            scale = np.abs(e) @ np.abs(L).T / sigma
            T = y
        else:
            ref, T, scale = reference(L, margins, nu, key, ctr0, n)
        for j in range(d):
            gain = np.abs(ref[:, j] / np.where(T[:, j] == 0, 1, T[:, j]))
            tol = 1e-12 * np.abs(ref[:, j]) + 1e-15 * scale[:, j] * np.maximum(gain, 1.0)
            assert np.all(np.abs(x[:, j] - ref[:, j]) <= tol), (nu, j)
