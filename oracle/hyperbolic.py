"""Oracle for the exponential -> hyperbolic recycling map -- TEST INFRASTRUCTURE ONLY.

Only ``tests/`` may import this module; the product library never does and
shares no code with it.

Sec. 8.1 (hyperbolic quantile from an exponential base): the target is the
hyperbolic density (location 0)

    f(x) = gamma / (2 alpha delta K_1(delta gamma)) exp(-alpha sqrt(delta^2 + x^2) + beta x),
    gamma = sqrt(alpha^2 - beta^2),  |beta| < alpha,  delta > 0,

and the base the two-sided exponential with the same split of mass at 0,

    f_0(v) = p_+ (alpha - beta) e^{-(alpha - beta) v}   (v > 0),
             p_- (alpha + beta) e^{(alpha + beta) v}    (v < 0),
    p_+ = int_0^inf f,  p_- = 1 - p_+ .

The recycling map is Q(v) = F^{-1}(G_0(v)) with G_0 the base CDF.  This
module computes it from those definitions: the tail and centre integrals of f
by composite 24-point Gauss-Legendre quadrature, normalised with the closed
form 2 alpha delta K_1(delta gamma) / gamma (scipy.special.kve), and inverted
by Brent's method.  The integrand is analytic except for the branch points of
sqrt(delta^2 + t^2) at t = +-i delta, so each panel is made no wider than its
distance from them, and no wider than 2 / (alpha + |beta|) (|g'| is at most
alpha + |beta|, so exp(g) changes by at most e^2 across a panel); on such
panels the 24-point rule is exact to rounding.  An infinite range stops once
a panel adds less than 1e-19 of the sum (the integrand then decays at least
like e^{-(alpha - |beta|) t}, and the rest is below that again).

For v >= 0 it solves P(X > Q) = p_+ e^{-(alpha - beta) v} in the upper tail,
or int_0^Q f = p_+ (1 - e^{-(alpha - beta) v}) near 0 (so that Q keeps its
relative accuracy as v -> 0); v < 0 uses the reflection
Q(v; beta) = -Q(-v; -beta).  Slow (a few ms per value) and plain.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import optimize, special

_GL_X, _GL_W = np.polynomial.legendre.leggauss(24)
# Brent's absolute tolerance: the smallest subnormal, so that only the relative
# tolerance counts even for roots near 1e-300 (v -> 0)
_XTOL = 5e-324


def _panel_integral(fn, lo, hi, t_off, delta, cap):
    """int_lo^hi fn(u) du (hi may be inf) by 24-point Gauss-Legendre on
    panels no wider than the distance from the panel start to the branch
    points u = -t_off +- i delta, and no wider than cap.  fn takes arrays."""
    total = 0.0
    a = lo
    while a < hi:
        w = min(math.hypot(a + t_off, delta), cap)
        b = min(a + w, hi)
        half = 0.5 * (b - a)
        part = half * float(np.dot(_GL_W, fn(0.5 * (a + b) + half * _GL_X)))
        total += part
        a = b
        if math.isinf(hi) and part <= 1e-19 * total:
            break
    return total


class Hyperbolic:
    def __init__(self, alpha: float, beta: float, delta: float):
        if not (abs(beta) < alpha and delta > 0):
            raise ValueError("need |beta| < alpha and delta > 0")
        self.alpha, self.beta, self.delta = float(alpha), float(beta), float(delta)
        self.gamma = math.sqrt(alpha * alpha - beta * beta)
        self.cap = 2.0 / (self.alpha + abs(self.beta))
        # log of the normalising constant Z = int exp(g) = 2 alpha delta K_1(delta gamma) / gamma
        dg = delta * self.gamma
        self.log_z = math.log(2 * alpha * delta / self.gamma) + math.log(special.kve(1, dg)) - dg
        self.p_plus = self._int_0_to(math.inf)
        # the other half by its own integral (1 - p_+ would lose digits when p_+ ~ 1)
        self.p_minus = _panel_integral(lambda t: np.exp(self.g_arr(-t) - self.log_z), 0.0, math.inf,
                                       0.0, self.delta, self.cap)

    # g(x) = -alpha sqrt(delta^2 + x^2) + beta x, and g(x + u) - g(x) without cancellation
    def g(self, x):
        return -self.alpha * math.hypot(self.delta, x) + self.beta * x

    def g_arr(self, x):
        return -self.alpha * np.hypot(self.delta, x) + self.beta * x

    def _dg(self, x, u):
        a, d = self.alpha, self.delta
        return u * (self.beta - a * (2 * x + u) / (np.hypot(d, x + u) + math.hypot(d, x)))

    def log_sf(self, x: float) -> float:
        """log P(X > x) for x >= 0."""
        val = _panel_integral(lambda u: np.exp(self._dg(x, u)), 0.0, math.inf, x, self.delta, self.cap)
        return self.g(x) - self.log_z + math.log(val)

    def _int_0_to(self, x: float) -> float:
        """int_0^x f (x >= 0, possibly inf)."""
        return _panel_integral(lambda t: np.exp(self.g_arr(t) - self.log_z), 0.0, x, 0.0, self.delta,
                               self.cap)

    def density(self, x: float) -> float:
        return math.exp(self.g(x) - self.log_z)

    def _q_right(self, v: float) -> float:
        """Q(v) for v >= 0 (upper half of both distributions)."""
        if v == 0.0:
            return 0.0
        if math.isinf(v):
            return math.inf
        r = self.alpha - self.beta
        c = -math.expm1(-r * v)                      # 1 - e^{-rv}, relative-accurate
        rtol = 4 * np.finfo(float).eps
        if c < 0.5:
            target = self.p_plus * c                  # int_0^Q f = p_+ (1 - e^{-rv})
            f = lambda q: self._int_0_to(q) - target
            hi = 2 * target / self.density(0.0)      # Q ~ target / f(0) near v = 0
            while f(hi) < 0:
                hi *= 2
            return optimize.brentq(f, 0.0, hi, xtol=_XTOL, rtol=rtol, maxiter=500)
        target = math.log(self.p_plus) - r * v        # log P(X > Q)
        f = lambda q: self.log_sf(q) - target
        hi = 1.0
        while f(hi) > 0:
            hi *= 2
        return optimize.brentq(f, 0.0, hi, xtol=_XTOL, rtol=rtol, maxiter=500)

    def quantile_map(self, v: float) -> float:
        if math.isnan(v):
            return math.nan
        if v >= 0:
            return self._q_right(v)
        mirror = self if self.beta == 0 else Hyperbolic(self.alpha, -self.beta, self.delta)
        return -mirror._q_right(-v)


def recycle_hyperbolic(alpha: float, beta: float, delta: float, v) -> np.ndarray:
    """x_i = Q(v_i) = F^{-1}(G_0(v_i)) for an array of two-sided exponential samples."""
    h = Hyperbolic(alpha, beta, delta)
    mirror = h if beta == 0 else Hyperbolic(alpha, -beta, delta)
    v = np.asarray(v, dtype=np.float64)
    out = np.empty_like(v)
    for i, x in enumerate(v.ravel()):
        if math.isnan(x):
            out.flat[i] = math.nan
        elif x >= 0:
            out.flat[i] = math.copysign(h._q_right(x), x)
        else:
            out.flat[i] = -mirror._q_right(-x)
    return out
