"""Pins of the t-copula oracle functions (Sec. 9), on the CPU.

* chi2_from_normal(nu, z) = F_{chi2(nu)}^{-1}(Phi(z)): closed forms at nu = 2
  (an exponential law: W = -2 log(1 - Phi(z))) and nu = 1 (the square of a
  normal: W = 2 erfinv(Phi(z))^2 from below, sqrt W = -Phi^{-1}((1-Phi(z))/2)
  from above), the incomplete gamma against mpmath at 40 digits, the far
  tails (z = +-8.3) against an mpmath root, scipy's gammaincinv in the bulk,
  and E W = nu by Gauss-Hermite quadrature over the normal score.
* t_to_normal(nu, t) = Phi^{-1}(F_nu(t)): closed forms at nu = 1
  (F = 1/2 + atan(t)/pi) and nu = 2 (F = 1/2 + t/(2 sqrt(t^2+2))), mpmath at
  extreme t, and the round trip through the pinned normal -> t oracle.
"""
import math

import mpmath as mp
import numpy as np
import pytest
from scipy import special

import oracle

Z = np.concatenate([np.linspace(-8.3, 8.3, 333), [-1e-3, 1e-3, -1e-8, 1e-8]])


def rel(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.abs(a / b - 1)


def test_chi2_nu2_closed_form():
    w = oracle.chi2_from_normal(2.0, Z)
    ref = -2.0 * special.log_ndtr(-Z)
    assert rel(w, ref).max() < 2e-14


def test_chi2_nu1_closed_form():
    w = oracle.chi2_from_normal(1.0, Z)
    lo = Z <= 0
    ref = np.empty_like(Z)
    ref[lo] = 2.0 * special.erfinv(special.ndtr(Z[lo])) ** 2
    ref[~lo] = special.ndtri(special.ndtr(-Z[~lo]) / 2.0) ** 2
    assert rel(w, ref).max() < 5e-13


@pytest.mark.parametrize("a", [0.375, 1.0, 2.0, 3.7, 50.0])
def test_incomplete_gamma_against_mpmath(a):
    """The prefactor a log x - x - lgamma(a + 1) cancels terms of size ~a log a,
    so the absolute error of log P grows like a ulp(a log a)."""
    mp.mp.dps = 40
    L = oracle.lib()
    tol = 4e-15 * max(1.0, a * math.log(a))
    for x in (1e-40, 1e-8, 0.3, a, a + 1.5, 3 * a + 10, 700.0):
        P = mp.gammainc(a, 0, x, regularized=True)
        Q = mp.gammainc(a, x, mp.inf, regularized=True)
        s = math.log(x)
        if P > 0:
            assert abs(L.orc_log_gamma_p(a, s) - float(mp.log(P))) < tol * max(1.0, abs(float(mp.log(P))))
        if Q > mp.mpf(10) ** -300:
            assert abs(L.orc_log_gamma_q(a, s) - float(mp.log(Q))) < tol * max(1.0, abs(float(mp.log(Q))))


@pytest.mark.parametrize("nu", [0.75, 3.3, 50.0])
def test_chi2_far_tails_against_mpmath(nu):
    mp.mp.dps = 40
    k = mp.mpf(nu) / 2
    for z in (-8.3, -5.0, 5.0, 8.3):
        u = mp.ncdf(z)
        if z < 0:
            f = lambda s: mp.log(mp.gammainc(k, 0, mp.exp(s), regularized=True)) - mp.log(u)
            s0 = (mp.log(u) + mp.loggamma(k + 1)) / k
        else:
            f = lambda s: mp.log(mp.gammainc(k, mp.exp(s), mp.inf, regularized=True)) - mp.log(mp.ncdf(-z))
            s0 = mp.log(k + z * z + 2 * z * mp.sqrt(k) + 1)
        s = mp.findroot(f, s0)
        ref = 2 * mp.exp(s)
        got = oracle.chi2_from_normal(nu, np.array([z]))[0]
        assert abs(got / float(ref) - 1) < 2e-13, (nu, z, got, ref)


@pytest.mark.parametrize("nu", [0.75, 1.3, 4.0, 12.0, 100.0])
def test_chi2_bulk_against_scipy_and_mean(nu):
    zb = np.linspace(-5, 5, 101)
    w = oracle.chi2_from_normal(nu, zb)
    ref = np.where(zb <= 0, 2 * special.gammaincinv(nu / 2, special.ndtr(zb)),
                   2 * special.gammainccinv(nu / 2, special.ndtr(-zb)))   # each side from its own tail
    assert rel(w, ref).max() < 1e-12
    # E W = nu: Gauss-Hermite (probabilists') over the normal score
    x, wt = np.polynomial.hermite_e.hermegauss(120)
    e = np.sum(wt * oracle.chi2_from_normal(nu, x)) / math.sqrt(2 * math.pi)
    assert abs(e / nu - 1) < 1e-6


def test_t_to_normal_closed_forms():
    t = np.concatenate([np.geomspace(0.1, 1e15, 200), -np.geomspace(0.1, 1e15, 50)])
    at = np.abs(t)
    g1 = oracle.t_to_normal(1.0, t)
    ref1 = -np.sign(t) * special.ndtri(np.arctan(1.0 / at) / np.pi)
    assert rel(g1, ref1).max() < 1e-13
    r = np.sqrt(at * at + 2)
    g2 = oracle.t_to_normal(2.0, t)
    ref2 = -np.sign(t) * special.ndtri(1.0 / (r * (r + at)))
    assert rel(g2, ref2).max() < 1e-13


@pytest.mark.parametrize("nu", [0.75, 2.5, 30.0])
def test_t_to_normal_round_trip_and_mpmath(nu):
    z = np.concatenate([np.linspace(-8.3, 8.3, 167), [1e-6, -1e-6]])
    t = oracle.recycle_t(nu, z)
    back = oracle.t_to_normal(nu, t)
    nz = z != 0
    assert np.abs(back - z).max() < 1e-13 and rel(back[nz], z[nz]).max() < 1e-12
    assert np.all(back[~nz] == 0)
    mp.mp.dps = 40
    for tv in (1e-7, 0.4, 3.0, 1e3, 1e20):
        x = mp.mpf(nu) / (nu + mp.mpf(tv) ** 2)
        p = mp.betainc(mp.mpf(nu) / 2, mp.mpf(1) / 2, 0, x, regularized=True) / 2      # P(T > t)
        if p < mp.mpf(10) ** -300:
            continue                     # outside the double range of the oracle's tail
        ref = -mp.sqrt(2) * mp.erfinv(2 * p - 1) if p > mp.mpf("1e-10") else None
        if ref is None:
            ref = mp.findroot(lambda w: mp.log(mp.ncdf(-w)) - mp.log(p), mp.sqrt(-2 * mp.log(p)))
        got = oracle.t_to_normal(nu, np.array([tv]))[0]
        assert abs(got / float(ref) - 1) < 2e-13, (nu, tv, got, ref)
