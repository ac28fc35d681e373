"""Target functions for the offline fits, in mpmath (30+ digits).

* ``q_exp(v)``  -- Q(v) = Phi^{-1}(1 - e^{-v}/2), the normal quantile in the
  exponential coordinate v = -log(2 min(u, 1-u)) (Sec. 6, Eq. for Q(v)).
* ``psi_t2(v)`` -- Psi(v) = Phi^{-1}((1 + v/sqrt(1+v^2))/2), the normal
  quantile in the scaled Student-t_2 coordinate v = |u - 1/2|/sqrt(u - u^2)
  (Sec. 7.3).
Both go through ``upper_probit(d)``, the w > 0 with 1 - Phi(w) = d, solved by
Newton's method on log erfc.
"""
import mpmath as mp


def upper_probit(d):
    """w >= 0 with erfc(w/sqrt2)/2 = d, for 0 < d <= 1/2."""
    d = mp.mpf(d)
    if d == mp.mpf(1) / 2:
        return mp.mpf(0)
    if d > mp.mpf("0.05"):
        return mp.sqrt(2) * mp.erfinv(1 - 2 * d)
    L = mp.log(d)
    w = mp.sqrt(-2 * L - mp.log(-2 * L * 2 * mp.pi))  # asymptotic start
    if w < 1:
        w = mp.mpf(1.5)
    for _ in range(100):
        x = w / mp.sqrt(2)
        g = mp.log(mp.erfc(x) / 2) - L
        lam = mp.sqrt(2 / mp.pi) * mp.exp(-x * x) / mp.erfc(x)  # phi/(1-Phi)
        dw = g / lam
        w += dw
        if abs(dw) < mp.mpf(10) ** (-mp.mp.dps + 5) * w:
            break
    return w


def q_exp(v):
    v = mp.mpf(v)
    if v == 0:
        return mp.mpf(0)
    if v < mp.mpf("1e-6"):
        # Phi^{-1}(1 - e^{-v}/2) = sqrt2 erfinv(1 - e^{-v}) = sqrt2 erfinv(-expm1(-v))
        return mp.sqrt(2) * mp.erfinv(-mp.expm1(-v))
    return upper_probit(mp.exp(-v) / 2)


def psi_t2(v):
    v = mp.mpf(v)
    if v == 0:
        return mp.mpf(0)
    r = mp.sqrt(1 + v * v)
    d = 1 / (2 * r * (r + v))          # 1 - (1 + v/r)/2, no cancellation
    if d > mp.mpf("0.05"):
        return mp.sqrt(2) * mp.erfinv(v / r)
    return upper_probit(d)
