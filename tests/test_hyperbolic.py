"""Exponential -> hyperbolic recycling (Sec. 8.1), on the CPU.

The oracle (oracle/hyperbolic.py: quadrature + Brent) is pinned to what the
paper and the mathematics fix: the normalising constant's closed form
2 alpha delta K_1(delta gamma)/gamma, the paper's slope Q'(0+) =
p_+ (alpha - beta) 2 (alpha delta / gamma) K_1(delta gamma) e^{alpha delta},
the delta -> 0 limit (the hyperbolic law becomes the base's asymmetric
Laplace law, so Q -> identity), the reflection Q(v; beta) = -Q(-v; -beta),
and the closed-form mean E X = beta delta K_2(delta gamma) / (gamma K_1(delta gamma))
recovered as the base expectation of Q.  The library's host-built tables
(qm_hyp_table_build), evaluated in numpy in the device's order, are then
checked against the oracle within 1e-12 relative.
"""
import math

import numpy as np
import pytest
from scipy import special

import paper_0901_0638_gb300 as qm
from oracle.hyperbolic import Hyperbolic, recycle_hyperbolic

PARAMS = [(1.0, 0.0, 1.0), (1.3, 0.4, 0.7), (2.0, -1.5, 0.05), (0.5, 0.2, 5.0), (1.0, 0.9, 2.0)]


def paper_slope(a, b, d, p_plus):
    g = math.sqrt(a * a - b * b)
    return p_plus * (a - b) * 2 * (a * d / g) * special.kv(1, d * g) * math.exp(a * d)


@pytest.mark.parametrize("a,b,d", PARAMS)
def test_oracle_normalisation_and_paper_slope(a, b, d):
    h = Hyperbolic(a, b, d)
    from scipy import integrate
    z = integrate.quad(lambda x: math.exp(h.g(x)), -math.inf, math.inf, epsabs=0, epsrel=1e-13, limit=400)[0]
    assert abs(z / math.exp(h.log_z) - 1) < 1e-12
    eps = 1e-7
    slope = (h.quantile_map(eps) - h.quantile_map(-eps)) / (2 * eps)   # one-sided slopes differ ...
    right = h.quantile_map(eps) / eps
    assert abs(right / paper_slope(a, b, d, h.p_plus) - 1) < 1e-5
    assert slope > 0


def test_oracle_delta_to_zero_is_identity():
    h = Hyperbolic(1.3, 0.4, 1e-9)
    for v in (1e-3, 0.3, 2.0, -1.5, 20.0, -7.0):
        assert abs(h.quantile_map(v) / v - 1) < 1e-7


def test_oracle_reflection_and_symmetry():
    a, b, d = 1.3, 0.4, 0.7
    v = np.array([0.01, 0.7, 3.0, 11.0])
    assert np.allclose(recycle_hyperbolic(a, b, d, -v), -recycle_hyperbolic(a, -b, d, v), rtol=1e-14, atol=0)
    h = Hyperbolic(1.0, 0.0, 1.0)
    assert abs(h.p_plus - 0.5) < 1e-15


def test_oracle_mean_closed_form():
    a, b, d = 1.3, 0.4, 0.7
    h = Hyperbolic(a, b, d)
    g = math.sqrt(a * a - b * b)
    mean = b * d * special.kv(2, d * g) / (g * special.kv(1, d * g))
    # E Q(V) over the base, by Gauss-Laguerre on each half-line
    xs, ws = np.polynomial.laguerre.laggauss(80)
    rp, rm = a - b, a + b
    qp = recycle_hyperbolic(a, b, d, xs / rp)
    qm_ = recycle_hyperbolic(a, b, d, -xs / rm)
    e = h.p_plus * np.sum(ws * qp) + h.p_minus * np.sum(ws * qm_)
    assert abs(e - mean) < 1e-9 * max(1.0, abs(mean))


def evaluate(tables, v):
    """The device's evaluation: binade segments of |v|, series about 0 below."""
    right, left, e_max, _ = tables
    v = np.asarray(v, dtype=np.float64)
    a = np.abs(v)
    out = np.empty_like(a)
    for side, mask in ((right, v >= 0), (left, v < 0)):
        if not mask.any():
            continue
        em = e_max[0] if side is right else e_max[1]
        aa = a[mask]
        m, E = np.frexp(aa)                  # aa = m 2^E, m in [0.5, 1)
        E = np.where(aa == 0, -1075, E - 1)  # aa in [2^E, 2^(E+1)); 0 takes the series about 0
        res = np.empty_like(aa)
        central = E < qm.QM_HYP_E_MIN
        Ec = np.minimum(E, em)
        j = np.where(E > em, 31, np.floor((aa / np.ldexp(1.0, E) - 1) * 32).astype(int))
        c = np.ldexp(1 + (2 * j + 1) / 64.0, Ec)
        idx = np.where(central, 0, 1 + 32 * (Ec - qm.QM_HYP_E_MIN) + j)
        s = np.where(central, aa, aa - c)
        coef = side[idx]
        acc = np.zeros_like(aa)
        for k in range(9, -1, -1):
            acc = acc * s + coef[:, k]
        res[:] = acc
        out[mask] = res
    return np.copysign(out, v)


def base_samples(a, b, p_plus, n, rng):
    """Two-sided exponential samples of the base law, plus edge magnitudes."""
    side = rng.random(n) < p_plus
    v = np.where(side, rng.exponential(1 / (a - b), n), -rng.exponential(1 / (a + b), n))
    extra = np.array([1e-300, 1e-20, 2.0**-30, 1e-9, 1e-3, 0.25, 1.0, 5.0, 30.0, 120.0])
    return np.concatenate([v, extra, -extra, [0.0, 700 / (a - b), -700 / (a + b)]])


@pytest.mark.parametrize("a,b,d", PARAMS)
def test_host_tables_against_the_oracle(a, b, d):
    tables = qm.qm_hyp_table_build(a, b, d)
    info = tables[3]
    h = Hyperbolic(a, b, d)
    assert abs(info[0] / h.p_plus - 1) < 1e-14 and abs(info[1] / h.p_minus - 1) < 1e-14
    assert abs(info[2] / paper_slope(a, b, d, h.p_plus) - 1) < 1e-13
    rng = np.random.default_rng(int(1000 * abs(a + 3 * b + 7 * d)))
    v = base_samples(a, b, h.p_plus, 400, rng)
    x = evaluate(tables, v)
    w = recycle_hyperbolic(a, b, d, v)
    nz = w != 0
    rel = np.abs(x[nz] / w[nz] - 1)
    assert rel.max() < 1e-12, (v[nz][np.argmax(rel)], rel.max())
    assert np.all(x[~nz] == 0)


def test_parameter_validation():
    for args, st in [((1.0, 1.0, 1.0), qm.QM_ERR_INVALID), ((1.0, 0.0, -1.0), qm.QM_ERR_INVALID),
                     ((1.0, 0.9999, 1.0), qm.QM_ERR_UNSUPPORTED), ((1.0, 0.0, 1e-6), qm.QM_ERR_UNSUPPORTED)]:
        with pytest.raises(qm.QMError) as e:
            qm.qm_hyp_table_build(*args)
        assert e.value.status == st
