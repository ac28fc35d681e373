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
by adaptive quadrature (scipy.integrate.quad), normalised with the closed
form 2 alpha delta K_1(delta gamma) / gamma (scipy.special.kv), and inverted
by Brent's method.  For v >= 0 it solves P(X > Q) = p_+ e^{-(alpha - beta) v}
in the upper tail, or int_0^Q f = p_+ (1 - e^{-(alpha - beta) v}) near 0 (so
that Q keeps its relative accuracy as v -> 0); v < 0 uses the reflection
Q(v; beta) = -Q(-v; -beta).  Slow (a few ms per value) and plain.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import integrate, optimize, special

_QUAD = dict(epsabs=0.0, epsrel=1.2e-14, limit=400)   # quad accepts >= 50 eps


class Hyperbolic:
    def __init__(self, alpha: float, beta: float, delta: float):
        if not (abs(beta) < alpha and delta > 0):
            raise ValueError("need |beta| < alpha and delta > 0")
        self.alpha, self.beta, self.delta = float(alpha), float(beta), float(delta)
        self.gamma = math.sqrt(alpha * alpha - beta * beta)
        # log of the normalising constant Z = int exp(g) = 2 alpha delta K_1(delta gamma) / gamma
        dg = delta * self.gamma
        self.log_z = math.log(2 * alpha * delta / self.gamma) + math.log(special.kve(1, dg)) - dg
        self.p_plus = self._int_0_to(math.inf)
        # the other half by its own integral (1 - p_+ would lose digits when p_+ ~ 1)
        val, _ = integrate.quad(lambda t: math.exp(self.g(-t) - self.log_z), 0.0, math.inf, **_QUAD)
        self.p_minus = val

    # g(x) = -alpha sqrt(delta^2 + x^2) + beta x, and g(x + u) - g(x) without cancellation
    def g(self, x):
        return -self.alpha * math.hypot(self.delta, x) + self.beta * x

    def _dg(self, x, u):
        a, d = self.alpha, self.delta
        return u * (self.beta - a * (2 * x + u) / (math.hypot(d, x + u) + math.hypot(d, x)))

    def log_sf(self, x: float) -> float:
        """log P(X > x) for x >= 0."""
        val, _ = integrate.quad(lambda u: math.exp(self._dg(x, u)), 0.0, math.inf, **_QUAD)
        return self.g(x) - self.log_z + math.log(val)

    def _int_0_to(self, x: float) -> float:
        """int_0^x f (x >= 0, possibly inf)."""
        val, _ = integrate.quad(lambda t: math.exp(self.g(t) - self.log_z), 0.0, x, **_QUAD)
        return val

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
            return optimize.brentq(f, 0.0, hi, xtol=1e-300, rtol=rtol, maxiter=500)
        target = math.log(self.p_plus) - r * v        # log P(X > Q)
        f = lambda q: self.log_sf(q) - target
        hi = 1.0
        while f(hi) > 0:
            hi *= 2
        return optimize.brentq(f, 0.0, hi, xtol=1e-300, rtol=rtol, maxiter=500)

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
