"""Gaussian copula with recycled marginals (Sec. 9 folding): the device
samples against a numpy reference built from the oracle (Philox words ->
oracle normals -> L eps -> oracle Student-t map), and the normal-score
correlation against L L^T."""
import numpy as np
import pytest
import torch

import oracle
import paper_0901_0638_gb300 as qm

pytestmark = pytest.mark.gpu
DEV = "cuda"


def reference(L, margins, key, ctr0, n):
    d = L.shape[0]
    nb = (d + 1) // 2
    w = oracle.philox_stream(key, ctr0, 4 * nb * n).astype(np.uint64).reshape(n, nb, 4)
    m = np.stack([((w[..., 0] >> 11) << 32) | w[..., 1], ((w[..., 2] >> 11) << 32) | w[..., 3]], axis=-1)
    m = m.reshape(n, 2 * nb)[:, :d]
    upper = m >= 2**52
    dd = (np.where(upper, 2**53 - 1 - m, m).astype(np.float64) + 0.5) * 2.0**-53
    eps = oracle.probit(dd.ravel()).reshape(dd.shape)
    eps = np.where(upper, -eps, eps)
    sigma = np.sqrt((L * L).sum(axis=1))            # rows normalised: the copula of the correlation
    y = eps @ L.T / sigma
    x = np.empty_like(y)
    for j, (kind, nu) in enumerate(margins):
        x[:, j] = oracle.recycle_t(nu, y[:, j]) if kind == qm.QM_DIST_STUDENT_T else y[:, j]
    scale = np.abs(eps) @ np.abs(L).T / sigma
    return x, y, scale


def test_copula_against_reference():
    rng = np.random.default_rng(9)
    d = 5
    A = rng.normal(size=(d, d))
    C = A @ A.T + d * np.eye(d)
    s = np.sqrt(np.diag(C))
    L = np.linalg.cholesky(C / np.outer(s, s))
    margins = [(qm.QM_DIST_NORMAL, 0.0), (qm.QM_DIST_STUDENT_T, 4.0), (qm.QM_DIST_STUDENT_T, 2.7),
               (qm.QM_DIST_NORMAL, 0.0), (qm.QM_DIST_STUDENT_T, 30.0)]
    c = qm.Copula(L, margins)
    n, key, ctr0 = 5003, 17, 8
    out = torch.empty(d * n, dtype=torch.float64, device=DEV)
    c.sample(key, ctr0, out, n)
    torch.cuda.synchronize()
    x = out.cpu().numpy().reshape(d, n).T
    w, y, scale = reference(L, margins, key, ctr0, n)
    for j, (kind, nu) in enumerate(margins):
        slope = np.abs(w[:, j] / np.where(y[:, j] == 0, 1, y[:, j]))      # |Q(y)/y| ~ local gain
        tol = 1e-12 * np.abs(w[:, j]) + 1e-15 * scale[:, j] * np.maximum(slope, 1.0)
        assert np.all(np.abs(x[:, j] - w[:, j]) <= tol), (j, np.max(np.abs(x[:, j] - w[:, j]) - tol))
    c.close()


def test_copula_correlation_of_normal_scores():
    R = np.array([[1.0, 0.6, 0.3], [0.6, 1.0, 0.5], [0.3, 0.5, 1.0]])
    L = np.linalg.cholesky(R)
    c = qm.Copula(L, [(qm.QM_DIST_NORMAL, 0.0)] * 3)
    n = 1 << 20
    out = torch.empty(3 * n, dtype=torch.float64, device=DEV)
    c.sample(5, 0, out, n)
    x = out.view(3, n)
    emp = torch.corrcoef(x).cpu().numpy()
    sd = (1 - R**2) / np.sqrt(n)
    assert np.all(np.abs(emp - R) <= 5 * sd + 1e-12)
    assert abs(float(x.mean())) < 5 / np.sqrt(3 * n)
    c.close()


def test_copula_argument_errors():
    eye = np.eye(3)
    with pytest.raises(qm.QMError) as e:
        qm.Copula(np.triu(np.ones((3, 3))), [(qm.QM_DIST_NORMAL, 0.0)] * 3)   # not lower triangular
    assert e.value.status == qm.QM_ERR_INVALID
    with pytest.raises(qm.QMError) as e:
        qm.Copula(np.eye(17), [(qm.QM_DIST_NORMAL, 0.0)] * 17)
    assert e.value.status == qm.QM_ERR_INVALID
    with pytest.raises(qm.QMError) as e:
        qm.Copula(eye, [(qm.QM_DIST_NORMAL, 0.0), (qm.QM_DIST_STUDENT_T, 0.5), (qm.QM_DIST_NORMAL, 0.0)])
    assert e.value.status == qm.QM_ERR_UNSUPPORTED
    with pytest.raises(qm.QMError) as e:
        qm.Copula(eye, [(qm.QM_DIST_EXPONENTIAL, 0.0)] * 3)
    assert e.value.status == qm.QM_ERR_UNSUPPORTED
