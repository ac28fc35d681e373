/*
 * orc.c -- CPU FP64 oracle (TEST INFRASTRUCTURE ONLY; see orc.h).
 *
 * Plain, slow, obviously correct.  Nothing here is tuned; the only goal is a
 * value a reader can check against the definitions by eye.
 */
#define _GNU_SOURCE
#include "orc.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <unistd.h>

#define ORC_SQRT_2_OVER_PI 0.79788456080286535588 /* sqrt(2/pi) */
#define ORC_LN2_HI 0.69314718055994528623          /* ln 2 rounded        */
#define ORC_LN2_LO 2.3190468138462996154e-17       /* ln 2 - ORC_LN2_HI   */

/* ------------------------------------------------------------------------
 * erf and erfc
 * ---------------------------------------------------------------------- */

/* Maclaurin series, A&S 7.1.5:
 *   erf(x) = 2/sqrt(pi) * sum_{n>=0} (-1)^n x^(2n+1) / (n! (2n+1)).
 * Used for |x| < 0.75, where the alternating sum loses under one bit.      */
static double erf_series(double x)
{
    double x2 = x * x;
    double term = x; /* (-1)^n x^(2n+1) / n! */
    double sum = x;
    for (int n = 1; n < 200; ++n) {
        term *= -x2 / n;
        double add = term / (2 * n + 1);
        sum += add;
        if (fabs(add) < 1e-18 * fabs(sum)) break;
    }
    return M_2_SQRTPI * sum;
}

/* erfcx(x) = exp(x^2) erfc(x) for x >= 0.75 from the even contraction of the
 * Laplace continued fraction (A&S 7.1.14):
 *   erfc(x) = 2x exp(-x^2)/sqrt(pi) /
 *             (b0 - a1/(b1 - a2/(b2 - ...))),
 *   b_n = 2x^2 + 1 + 4n,  a_n = (2n-1)(2n).
 * Evaluated backwards from a fixed depth N that over-covers the forward
 * convergence count (about 95 terms at x = 1, 28 at x = 2).              */
static double erfcx_cf(double x)
{
    double x2 = 2.0 * x * x;
    int N = 60 + (int)(400.0 / (x * x));
    if (N > 4000) N = 4000;
    double T = x2 + 1.0 + 4.0 * N;
    for (int n = N; n >= 1; --n) {
        double a = (2.0 * n - 1.0) * (2.0 * n);
        T = (x2 + 1.0 + 4.0 * (n - 1)) - a / T;
    }
    return M_2_SQRTPI * x / T;
}

/* exp(-w^2/2) with w^2 split exactly into hi + lo (fma), so that the rounding
 * of w^2 does not enter the exponent.                                      */
static double exp_neg_half_sq(double w)
{
    double h = w * w;
    double l = fma(w, w, -h);
    return exp(-0.5 * h) * (1.0 - 0.5 * l);
}

double orc_erfcx(double x)
{
    if (isnan(x)) return x;
    if (x < 0.75) {
        /* exp(x^2) (1 - erf(x)); only the x >= 0 range is promised. */
        double h = x * x, l = fma(x, x, -h);
        return exp(h) * (1.0 + l) * (1.0 - erf_series(x));
    }
    return erfcx_cf(x);
}

double orc_erf(double x)
{
    if (isnan(x)) return x;
    double a = fabs(x);
    if (a < 0.75) return erf_series(x);
    if (a > 6.5) return copysign(1.0, x);
    double h = a * a, l = fma(a, a, -h);
    double c = exp(-h) * (1.0 - l) * erfcx_cf(a);
    return copysign(1.0 - c, x);
}

double orc_erfc(double x)
{
    if (isnan(x)) return x;
    if (x < 0.0) return 2.0 - orc_erfc(-x);
    if (x < 0.75) return 1.0 - erf_series(x);
    if (x > 27.3) return 0.0;
    double h = x * x, l = fma(x, x, -h);
    return exp(-h) * (1.0 - l) * erfcx_cf(x);
}

/* 1 - Phi(w) = erfc(w/sqrt2)/2.  In the tail the factor exp(-w^2/2) is taken
 * with exact w^2; only the smooth continued-fraction factor sees the rounded
 * argument w/sqrt2.                                                        */
double orc_norm_sf(double w)
{
    if (isnan(w)) return w;
    if (w < 0.0) return 1.0 - orc_norm_sf(-w);
    double x = w * M_SQRT1_2;
    if (x < 0.75) return 0.5 * (1.0 - erf_series(x));
    if (w > 40.0) return 0.0;
    return 0.5 * exp_neg_half_sq(w) * erfcx_cf(x);
}

double orc_norm_cdf(double w) { return orc_norm_sf(-w); }

double orc_log_norm_sf(double w)
{
    if (isnan(w)) return w;
    if (w < 0.0) return log1p(-orc_norm_sf(-w));
    double x = w * M_SQRT1_2;
    if (x < 0.75) return log(0.5 * (1.0 - erf_series(x)));
    double h = w * w, l = fma(w, w, -h);
    return (-0.5 * h - 0.5 * l) + log(0.5 * erfcx_cf(x));
}

/* ------------------------------------------------------------------------
 * Normal quantile Phi^{-1}
 * ---------------------------------------------------------------------- */

/* Root w in [0, 0.7] of erf(w/sqrt2) = t for t in [0, 1/2]: the centre form,
 * which keeps full relative accuracy as w -> 0 (t = |2u - 1| is exact).     */
double orc_probit_centre(double t)
{
    if (t == 0.0) return 0.0;
    double lo = 0.0, hi = 0.7;
    double w = t * 1.2533141373155002512; /* t sqrt(pi/2), the slope at 0 */
    if (!(w > lo && w < hi)) w = 0.5 * (lo + hi);
    for (int it = 0; it < 200; ++it) {
        double f = erf_series(w * M_SQRT1_2) - t;
        if (f > 0) hi = w; else lo = w;
        if (f == 0) return w;
        double fp = ORC_SQRT_2_OVER_PI * exp(-0.5 * w * w);
        double wn = w - f / fp;
        if (!(wn > lo && wn < hi)) wn = 0.5 * (lo + hi);
        if (fabs(wn - w) <= 1e-17 * w || hi - lo <= 4e-17 * hi) { w = wn; break; }
        w = wn;
    }
    return w;
}

/* Root w >= 0.6 of log(1 - Phi(w)) = L for L <= log(1/4): the tail form.
 * Working in log space keeps the equation well scaled down to the smallest
 * subnormal and makes Newton's iteration nearly linear.                   */
double orc_probit_tail_log(double L)
{
    double lo = 0.6, hi = 40.0;
    double a = -2.0 * L;
    double w = sqrt(fmax(a - log(2.0 * M_PI * a), 0.49));
    if (!(w > lo && w < hi)) w = 0.5 * (lo + hi);
    for (int it = 0; it < 300; ++it) {
        double g = orc_log_norm_sf(w) - L; /* decreasing in w */
        if (g > 0) lo = w; else hi = w;
        if (g == 0) return w;
        double x = w * M_SQRT1_2;
        double lam = (x < 0.75)
            ? (ORC_SQRT_2_OVER_PI * 0.5 * exp(-0.5 * w * w)) /
                  (0.5 * (1.0 - erf_series(x)))
            : ORC_SQRT_2_OVER_PI / erfcx_cf(x); /* phi(w) / (1 - Phi(w)) */
        double wn = w + g / lam;
        if (!(wn > lo && wn < hi)) wn = 0.5 * (lo + hi);
        if (fabs(wn - w) <= 1e-17 * w || hi - lo <= 4e-17 * hi) { w = wn; break; }
        w = wn;
    }
    return w;
}

/* Phi^{-1}(u).  d = min(u, 1-u) is exact (1 - u is exact for u >= 1/2);
 * d >= 1/4 solves the centre form on t = |2u - 1| (exact), d < 1/4 the tail
 * form on log d.  Phi^{-1}(0) = -inf, Phi^{-1}(1) = +inf, NaN outside [0,1].*/
double orc_probit(double u)
{
    if (isnan(u) || u < 0.0 || u > 1.0) return NAN;
    if (u == 0.0) return -INFINITY;
    if (u == 1.0) return INFINITY;
    double s = (u > 0.5) ? 1.0 : -1.0;
    double d = (u > 0.5) ? 1.0 - u : u;
    if (d >= 0.25) {
        double t = fabs(2.0 * u - 1.0);
        if (t == 0.0) return 0.0;
        return s * orc_probit_centre(t);
    }
    return s * orc_probit_tail_log(log(d));
}

/* ------------------------------------------------------------------------
 * Student t
 * ---------------------------------------------------------------------- */

static double lbeta(double a, double b)
{
    return lgamma(a) + lgamma(b) - lgamma(a + b);
}

/* Continued fraction of DLMF 8.17.22 by the modified Lentz method:
 *   I_x(a,b) = x^a (1-x)^b / (a B(a,b)) * 1/(1+ d1/(1+ d2/(1+ ...))),
 *   d_{2m+1} = -(a+m)(a+b+m) x / ((a+2m)(a+2m+1)),
 *   d_{2m}   =  m (b-m) x / ((a+2m-1)(a+2m)).
 * Returns the continued-fraction value 1/(1+ d1/(1+ ...)).                */
static double ibeta_cf(double a, double b, double x)
{
    const double tiny = 1e-300;
    double f = 1.0, C = 1.0, D = 0.0;
    for (int k = 1; k < 20000; ++k) {
        int m = k / 2;
        double dk = (k & 1)
            ? -(a + m) * (a + b + m) * x / ((a + 2 * m) * (a + 2 * m + 1))
            : m * (b - m) * x / ((a + 2 * m - 1) * (a + 2 * m));
        D = 1.0 + dk * D;
        if (fabs(D) < tiny) D = tiny;
        C = 1.0 + dk / C;
        if (fabs(C) < tiny) C = tiny;
        D = 1.0 / D;
        double delta = C * D;
        f *= delta;
        if (fabs(delta - 1.0) < 1e-17) break;
    }
    return 1.0 / f;
}

/* log I_x(a,b) for x in the fast-converging range x < (a+1)/(a+b+2). */
static double log_ibeta_direct(double a, double b, double x, double logx)
{
    return a * logx + b * log1p(-x) - lbeta(a, b) - log(a) +
           log(ibeta_cf(a, b, x));
}

double orc_ibeta(double a, double b, double x)
{
    if (isnan(x)) return x;
    if (x <= 0.0) return 0.0;
    if (x >= 1.0) return 1.0;
    if (x < (a + 1.0) / (a + b + 2.0))
        return exp(log_ibeta_direct(a, b, x, log(x)));
    return 1.0 - exp(log_ibeta_direct(b, a, 1.0 - x, log1p(-x)));
}

/* P(T > t) = I_{nu/(nu+t^2)}(nu/2, 1/2) / 2 for t >= 0 (Sec. 3.1 density). */
double orc_t_sf(double nu, double t)
{
    if (t < 0.0) return 1.0 - orc_t_sf(nu, -t);
    double x = nu / (nu + t * t);
    return 0.5 * orc_ibeta(0.5 * nu, 0.5, x);
}

/* gamma = Q'(0) = sqrt(nu/2) Gamma(nu/2) / Gamma((nu+1)/2) (Sec. 3.1). */
double orc_t_gamma(double nu)
{
    return exp(0.5 * log(0.5 * nu) + lgamma(0.5 * nu) - lgamma(0.5 * (nu + 1)));
}

/* Increasing function g(s) = log I_{e^s}(a, b) and its derivative, for the
 * Newton solve in s = log x.                                              */
static double log_ibeta_s(double a, double b, double s, double* dds)
{
    double x = exp(s);
    double lg;
    if (x < (a + 1.0) / (a + b + 2.0)) {
        lg = log_ibeta_direct(a, b, x, s);
    } else {
        double upper = exp(log_ibeta_direct(b, a, -expm1(s), log1p(-x)));
        lg = log1p(-upper);
    }
    /* d/ds log I = x f_beta(x) / I, f_beta = x^{a-1}(1-x)^{b-1}/B(a,b). */
    *dds = exp(a * s + (b - 1.0) * log1p(-x) - lbeta(a, b) - lg);
    return lg;
}

/* Root s <= 0 of log I_{e^s}(a, b) = target (target <= 0). */
static double solve_log_ibeta(double a, double b, double target, double s0)
{
    double lo = -2000.0, hi = 0.0;
    double s = s0;
    if (!(s > lo && s < hi)) s = -1.0;
    for (int it = 0; it < 400; ++it) {
        double d;
        double g = log_ibeta_s(a, b, s, &d) - target; /* increasing in s */
        if (g > 0) hi = s; else lo = s;
        if (g == 0) return s;
        double sn = s - g / d;
        if (!(sn > lo && sn < hi) || !isfinite(sn)) sn = 0.5 * (lo + hi);
        if (fabs(sn - s) <= 1e-16 * fmax(1.0, fabs(s)) || hi - lo < 1e-15) {
            s = sn;
            break;
        }
        s = sn;
    }
    return s;
}

/* Q(z) = F_nu^{-1}(Phi(z)), Sec. 3 (the normal -> Student t recycling map).
 * For z > 0 with p = 1 - Phi(z):
 *   p <  1/4: tail form,   solve I_x(nu/2, 1/2) = 2p for x = nu/(nu+t^2);
 *   p >= 1/4: centre form, solve I_y(1/2, nu/2) = erf(z/sqrt2) for
 *             y = t^2/(nu+t^2).
 * For |z| < 1e-9 the map is its centre slope t = gamma z (Sec. 3.1); the
 * next term is c_1 z^3, below 1e-17 relative there.  Odd in z.           */
double orc_recycle_normal_to_t(double nu, double z)
{
    if (isnan(z) || !(nu > 0.0)) return NAN;
    if (z == 0.0) return z;
    if (isinf(z)) return z;
    double az = fabs(z), sg = copysign(1.0, z);
    if (az < 1e-9) return sg * orc_t_gamma(nu) * az;
    double p = orc_norm_sf(az);
    double a = 0.5 * nu;
    if (p < 0.25) {
        double target = orc_log_norm_sf(az) + M_LN2; /* log(2p) */
        /* Leading tail behaviour I_x ~ x^a / (a B): start guess. */
        double s0 = (target + lbeta(a, 0.5) + log(a)) / a;
        if (s0 > -1e-3) s0 = -1e-3;
        double s = solve_log_ibeta(a, 0.5, target, s0);
        /* t = sqrt(nu (1-x)/x) = sqrt(nu (1-x)) exp(-s/2), 1-x = -expm1(s) */
        return sg * sqrt(nu * -expm1(s)) * exp(-0.5 * s);
    } else {
        double c = orc_erf(az * M_SQRT1_2);
        double target = log(c);
        double s0 = 2.0 * log(orc_t_gamma(nu) * az) - log(nu);
        if (s0 > -1e-3) s0 = -1e-3;
        double s = solve_log_ibeta(0.5, a, target, s0);
        double y = exp(s);
        return sg * sqrt(nu * y / (1.0 - y));
    }
}

/* ------------------------------------------------------------------------
 * Exponential background: Q(x) = Phi^{-1}(1 - exp(-x)), x >= 0
 * (Sec. 2.3, Sec. 6).  With u = 1 - e^{-x}:
 *   u >= 3/4 (x >= ln 4):   right tail, log(1-u) = -x exactly;
 *   u <= 1/4 (x <= ln 4/3): left tail,  d = u = -expm1(-x);
 *   otherwise centre, t = |2u - 1| = |expm1(ln 2 - x)|, ln 2 split hi+lo.
 * ---------------------------------------------------------------------- */
double orc_recycle_exp_to_normal(double x)
{
    if (isnan(x) || x < 0.0) return NAN;
    if (x == 0.0) return -INFINITY;
    if (isinf(x)) return INFINITY;
    if (x >= 1.3862943611198906) return orc_probit_tail_log(-x);
    if (x <= 0.28768207245178093) return -orc_probit_tail_log(log(-expm1(-x)));
    double v = (ORC_LN2_HI - x) + ORC_LN2_LO;
    double t = fabs(expm1(v));
    if (t == 0.0) return 0.0;
    double w = orc_probit_centre(t);
    return (v < 0.0) ? w : -w;
}

/* ------------------------------------------------------------------------
 * Chi-squared and the t -> normal map, for the t copula (Sec. 9).
 * ---------------------------------------------------------------------- */

/* log P(a, x) and log Q(a, x), the regularised incomplete gamma functions,
 * with x = e^s given by its logarithm (so x may lie far below the double
 * range).  Series, DLMF 8.7.1:
 *   P(a,x) = x^a e^{-x} / Gamma(a+1) * sum_{n>=0} x^n / ((a+1)...(a+n)),
 * for x < a + 1; otherwise the continued fraction of DLMF 8.9.2,
 *   Q(a,x) = x^a e^{-x} / Gamma(a) * 1/(x+1-a- 1(1-a)/(x+3-a- 2(2-a)/(...))),
 * by the modified Lentz method.  Each returns the log of its own function;
 * the complement is taken in log space.                                    */
static double log_gamma_p_series(double a, double s)
{
    const double x = exp(s);
    double term = 1.0, sum = 1.0;
    for (int n = 1; n < 100000; ++n) {
        term *= x / (a + n);
        sum += term;
        if (term < 1e-18 * sum) break;
    }
    return a * s - x - lgamma(a + 1.0) + log(sum);
}

static double log_gamma_q_cf(double a, double s)
{
    const double x = exp(s), tiny = 1e-300;
    double b = x + 1.0 - a;
    double C = 1.0 / tiny, D = 1.0 / b, f = D;
    for (int n = 1; n < 100000; ++n) {
        const double an = -n * (n - a);
        b += 2.0;
        D = an * D + b;
        if (fabs(D) < tiny) D = tiny;
        C = b + an / C;
        if (fabs(C) < tiny) C = tiny;
        D = 1.0 / D;
        const double delta = C * D;
        f *= delta;
        if (fabs(delta - 1.0) < 1e-17) break;
    }
    return a * s - x - lgamma(a) + log(f);
}

double orc_log_gamma_p(double a, double s)
{
    if (exp(s) < a + 1.0) return log_gamma_p_series(a, s);
    return log1p(-exp(log_gamma_q_cf(a, s)));
}

double orc_log_gamma_q(double a, double s)
{
    if (exp(s) < a + 1.0) return log1p(-exp(log_gamma_p_series(a, s)));
    return log_gamma_q_cf(a, s);
}

/* W = F^{-1}(Phi(z)) for W ~ chi-squared with nu degrees of freedom
 * (Gamma(nu/2) in x = W/2).  z <= 0 solves log P(nu/2, x) = log Phi(z),
 * z > 0 solves log Q(nu/2, x) = log(1 - Phi(z)), for s = log x by bisection
 * with Newton steps; both sides are relative-accurate far into the tails.
 * d log P / ds = x f(x) / P and d log Q / ds = -x f(x) / Q, with
 * x f(x) = x^a e^{-x} / Gamma(a).                                          */
double orc_chi2_from_normal(double nu, double z)
{
    if (isnan(z) || !(nu > 0.0)) return NAN;
    if (z == -INFINITY) return 0.0;
    if (z == INFINITY) return INFINITY;
    const double a = 0.5 * nu;
    const int lower = z <= 0.0;
    const double target = lower ? orc_log_norm_sf(-z) : orc_log_norm_sf(z);
    double lo = -3000.0, hi = 12.0;
    /* start: the leading term of the side being solved */
    double s = lower ? (target + lgamma(a + 1.0)) / a : log(a + 4.0 * z * z + 1.0);
    if (!(s > lo && s < hi)) s = 0.5 * (lo + hi);
    for (int it = 0; it < 400; ++it) {
        const double lp = lower ? orc_log_gamma_p(a, s) : orc_log_gamma_q(a, s);
        const double g = lower ? lp - target : target - lp;   /* increasing in s */
        if (g == 0.0) break;
        if (g > 0.0) hi = s; else lo = s;
        const double dlog = exp(a * s - exp(s) - lgamma(a) - lp);   /* |d lp / ds| */
        double sn = s - g / dlog;
        if (!(sn > lo && sn < hi)) sn = 0.5 * (lo + hi);
        if (fabs(sn - s) <= 1e-16 * fmax(1.0, fabs(s)) || hi - lo <= 1e-16 * fmax(1.0, fabs(hi))) {
            s = sn;
            break;
        }
        s = sn;
    }
    return 2.0 * exp(s);
}

/* G(t) = Phi^{-1}(F_nu(t)), the Student t -> normal map (the inverse of
 * orc_recycle_normal_to_t).  Odd in t.  With p = P(T > |t|):
 * p < 1/4: tail form -Phi^{-1}(p) from log p;
 * otherwise the centre form: 2 F(|t|) - 1 = I_y(1/2, nu/2), y = t^2/(nu+t^2),
 * and |G| solves erf(|G|/sqrt2) = that.  Domain: P(T > |t|) a normal double
 * (|G| below about 37.5).                                                  */
double orc_t_to_normal(double nu, double t)
{
    if (isnan(t) || !(nu > 0.0)) return NAN;
    if (t == 0.0) return t;
    if (isinf(t)) return t;
    const double at = fabs(t), sg = copysign(1.0, t);
    const double p = orc_t_sf(nu, at);
    if (p < 0.25) return sg * orc_probit_tail_log(log(p));
    const double y = at * at / (nu + at * at);
    return sg * orc_probit_centre(orc_ibeta(0.5, 0.5 * nu, y));
}

/* ------------------------------------------------------------------------
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).  One round maps the
 * counter (c0, c1, c2, c3) with round key (k0, k1) to
 *   (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)),
 * and the key is bumped by the Weyl constants between rounds.
 * ---------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                       uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)M0 * c0;
        uint64_t p1 = (uint64_t)M1 * c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += W0;
        k1 += W1;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

void orc_philox_stream(uint64_t seed, uint64_t first, size_t n, uint32_t* out)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (size_t j = 0; j < n; ++j) {
        uint64_t i = first + j;
        uint64_t blk = i >> 2;
        uint32_t ctr[4] = {(uint32_t)blk, (uint32_t)(blk >> 32), 0u, 0u};
        uint32_t o[4];
        orc_philox4x32_10(ctr, key, o);
        out[j] = o[i & 3];
    }
}

/* ------------------------------------------------------------------------
 * Array drivers: static block partition over POSIX threads.
 * ---------------------------------------------------------------------- */

typedef struct {
    int kind;
    double nu;
    const double* in;
    double* out;
    size_t lo, hi;
} job_t;

static void* run_job(void* arg)
{
    job_t* j = (job_t*)arg;
    for (size_t i = j->lo; i < j->hi; ++i) {
        double x = j->in[i];
        if (j->kind == 0) j->out[i] = orc_probit(x);
        else if (j->kind == 1) j->out[i] = orc_recycle_normal_to_t(j->nu, x);
        else j->out[i] = orc_recycle_exp_to_normal(x);
    }
    return NULL;
}

int orc_threads_used(int nthreads)
{
    if (nthreads > 0) return nthreads;
    long c = sysconf(_SC_NPROCESSORS_ONLN);
    return c > 0 ? (int)c : 1;
}

static int run_array(int kind, double nu, const double* in, double* out,
                     size_t n, int nthreads)
{
    int T = orc_threads_used(nthreads);
    if ((size_t)T > n) T = n > 0 ? (int)n : 1;
    if (T > 1024) T = 1024;
    pthread_t th[1024];
    job_t jobs[1024];
    for (int t = 0; t < T; ++t) {
        jobs[t].kind = kind;
        jobs[t].nu = nu;
        jobs[t].in = in;
        jobs[t].out = out;
        jobs[t].lo = n * (size_t)t / T;
        jobs[t].hi = n * (size_t)(t + 1) / T;
    }
    for (int t = 1; t < T; ++t) pthread_create(&th[t], NULL, run_job, &jobs[t]);
    run_job(&jobs[0]);
    for (int t = 1; t < T; ++t) pthread_join(th[t], NULL);
    return T;
}

int orc_probit_array(const double* u, double* z, size_t n, int nthreads)
{
    return run_array(0, 0.0, u, z, n, nthreads);
}

int orc_recycle_t_array(double nu, const double* z, double* t, size_t n,
                        int nthreads)
{
    return run_array(1, nu, z, t, n, nthreads);
}

int orc_recycle_exp_array(const double* x, double* z, size_t n, int nthreads)
{
    return run_array(2, 0.0, x, z, n, nthreads);
}
