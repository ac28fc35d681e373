"""Exponential -> hyperbolic recycling (Sec. 8.1), on the CPU.

The oracle (oracle/hyperbolic.py: quadrature + Brent) is pinned to what the
paper and the mathematics fix: the normalising constant's closed form
2 alpha delta K_1(delta gamma)/gamma, the paper's slope Q'(0+) =
p_+ (alpha - beta) 2 (alpha delta / gamma) K_1(delta gamma) e^{alpha delta},
the delta -> 0 limit (the hyperbolic law becomes the base's asymmetric
Laplace law, so Q -> identity), the reflection Q(v; beta) = -Q(-v; -beta),
and the closed-form mean E X = beta delta K_2(delta gamma) / (gamma K_1(delta gamma))
recovered as the base expectation of Q.  Every function of the oracle is
also pinned within 1e-13 (1e-14 for the integrals) to 30-digit mpmath
quadrature and Newton roots of the Sec. 8.1 definitions, in both tails out to
a base tail probability of 1e-300.  The library's host-built tables
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


# ---------------------------------------------------------------------------
# Pins against 30-digit mpmath, computed from the definitions of Sec. 8.1 with
# no shared step: the density exp(g)/Z integrated by tanh-sinh quadrature
# (mpmath.quad), Z by quadrature too (the oracle uses the K_1 closed form),
# and Q(v) as the root of G_0(v) = F(Q) by Newton's method on each side
# (v < 0 directly on the lower tail, not through the oracle's reflection).
# ---------------------------------------------------------------------------


class _MpHyperbolic:
    def __init__(self, mp, a, b, d):
        self.mp = mp
        self.a, self.b, self.d = mp.mpf(a), mp.mpf(b), mp.mpf(d)
        self.mode = self.d * self.b / mp.sqrt(self.a ** 2 - self.b ** 2)
        self.z = self.integral(-mp.inf, mp.inf)
        self.p_plus = self.integral(0, mp.inf) / self.z
        self.p_minus = self.integral(-mp.inf, 0) / self.z

    def g(self, t):
        return -self.a * self.mp.sqrt(self.d ** 2 + t ** 2) + self.b * t

    def integral(self, lo, hi, shift=0):
        """int_lo^hi exp(g(t) - shift) dt, split at the density's features."""
        mp = self.mp
        feats = [0, self.mode, self.d, -self.d, 4 * self.d, -4 * self.d]
        pts = [lo] + sorted(p for p in feats if lo < p < hi)
        for scale in (1 / (self.a - abs(self.b)), 10 / (self.a - abs(self.b))):
            if mp.isinf(hi) and not mp.isinf(pts[-1]):
                pts.append(pts[-1] + scale)
        if mp.isinf(lo) and not mp.isinf(pts[1] if len(pts) > 1 else hi):
            first = pts[1] if len(pts) > 1 else hi
            pts[1:1] = [first - 10 / (self.a - abs(self.b)), first - 1 / (self.a - abs(self.b))]
        pts.append(hi)
        total = mp.mpf(0)
        for lo_k, hi_k in zip(pts[:-1], pts[1:]):
            if mp.isinf(lo_k) or mp.isinf(hi_k):
                total += mp.quad(lambda t: mp.exp(self.g(t) - shift), [lo_k, hi_k])
            else:
                # on [0, 1]: tanh-sinh judges convergence in absolute terms,
                # so a tiny interval is rescaled to keep the integrand's size
                w = hi_k - lo_k
                total += w * mp.quad(lambda s: mp.exp(self.g(lo_k + w * s) - shift), [0, 1])
        return total

    def q(self, v, q0):
        """Q(v): Newton from q0 on log P(X > Q) = log(p_+) - (a - b) v (v > 0,
        tail), int_0^Q f = p_+ (1 - e^{-(a-b) v}) (v > 0, centre) and the
        mirrored equations for v < 0."""
        mp = self.mp
        v = mp.mpf(v)
        q = mp.mpf(q0)
        for _ in range(3):
            gq = self.g(q)
            if v > 0:
                c = -mp.expm1(-(self.a - self.b) * v)
                if c < 0.5:
                    F = self.integral(0, q) / self.z - self.p_plus * c
                    dF = mp.exp(gq) / self.z
                else:
                    tail = self.integral(q, mp.inf, gq)           # e^{-g(q)} int_q^inf e^g
                    F = gq + mp.log(tail) - mp.log(self.z) - (mp.log(self.p_plus) - (self.a - self.b) * v)
                    dF = -1 / tail
            else:
                c = -mp.expm1((self.a + self.b) * v)
                if c < 0.5:
                    F = self.integral(q, 0) / self.z - self.p_minus * c
                    dF = -mp.exp(gq) / self.z
                else:
                    tail = self.integral(-mp.inf, q, gq)
                    F = gq + mp.log(tail) - mp.log(self.z) - (mp.log(self.p_minus) + (self.a + self.b) * v)
                    dF = 1 / tail
            q = q - F / dF
        return q


@pytest.mark.parametrize("a,b,d", PARAMS)
def test_oracle_against_mpmath(a, b, d):
    """Every function of oracle/hyperbolic.py against 30-digit mpmath: log Z,
    p_+ and p_-, the centre integral, log P(X > x), and Q(v) on both sides from
    v = 1e-300 out to a base tail probability of 1e-300, within 1e-13."""
    mpmath = pytest.importorskip("mpmath")
    with mpmath.workdps(30):
        _check_against_mpmath(mpmath, a, b, d)


def _check_against_mpmath(mpmath, a, b, d):
    h = Hyperbolic(a, b, d)
    m = _MpHyperbolic(mpmath, a, b, d)
    assert abs(h.log_z - float(mpmath.log(m.z))) < 1e-14 * max(1.0, abs(h.log_z))
    assert abs(h.p_plus / float(m.p_plus) - 1) < 1e-14
    assert abs(h.p_minus / float(m.p_minus) - 1) < 1e-14
    r = a - b
    for x in (1e-200, 0.01 * d, d, 2.0 / r):
        ref = float(m.integral(0, mpmath.mpf(x)) / m.z)
        assert abs(h._int_0_to(x) / ref - 1) < 1e-14, x
    for x in (0.0, d, 3.0 / r, 30.0 / r, 300.0 / r):
        gx = m.g(mpmath.mpf(x))
        ref = float(gx + mpmath.log(m.integral(mpmath.mpf(x), mpmath.inf, gx) / m.z))
        assert abs(h.log_sf(x) - ref) < 1e-15 * abs(ref) + 1e-14, x
    # v > 0: centre branch (v -> 0) and tail branch out to p_+ e^{-r v} = 1e-300
    vs = [1e-300, 1e-12, 1e-3, 0.5 / r] + [math.log(h.p_plus / s) / r for s in (0.3, 1e-3, 1e-20, 1e-100, 1e-300)]
    # v < 0, the lower half directly (the oracle goes through its reflection)
    rl = a + b
    vs += [-1e-300, -1e-6, -0.3 / rl] + [-math.log(h.p_minus / s) / rl for s in (0.3, 1e-50, 1e-300)]
    for v in vs:
        got = h.quantile_map(v)
        ref = float(m.q(v, got))
        assert abs(got / ref - 1) < 1e-13, (v, got, ref)
    x = recycle_hyperbolic(a, b, d, np.array(vs + [0.0, math.inf, -math.inf, math.nan]))
    assert np.array_equal(x[: len(vs)], np.array([h.quantile_map(v) for v in vs]))
    assert x[len(vs)] == 0.0 and x[len(vs) + 1] == math.inf and x[len(vs) + 2] == -math.inf
    assert math.isnan(x[-1])


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
        with np.errstate(invalid="ignore", divide="ignore"):        # both branches are evaluated
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
