// qm_tcop_tables.cu -- host-built recycling tables of the t copula (Sec. 9).
//
// A t copula with nu degrees of freedom and correlation R draws
// T = (L eps) sqrt(nu / W), eps iid normal, W ~ chi-squared(nu), and maps each
// coordinate to its margin.  The paper notes that the trip through the unit
// hypercube folds into one recycling map per coordinate; two maps make that
// possible here, each tabulated per nu from its recycling ODE (Sec. 9 form,
// Q'' + H_0 Q' = H_1(Q) Q'^2, H_i = -(log f_i)'):
//
//   mixing variable  W(z) = F_chi2^{-1}(Phi(z))  (normal base, H_0 = z;
//                    chi-squared target, H_1(w) = -(k-1)/w + 1/2, k = nu/2):
//                    W W'' = -z W W' - (k-1) W'^2 + W W'^2 / 2,
//                    stored as L = log W, segments of width 1/16 on
//                    z in [-8.5, 8.5] (every 53-bit grid normal);
//   t -> normal      G(t) = Phi^{-1}(F_nu(t))  (Student-t base,
//                    H_0 = (nu+1) t / (nu + t^2); normal target, H_1 = G):
//                    (nu + t^2) G'' = -(nu+1) t G' + (nu + t^2) G G'^2;
//                    row 0 is its odd series about 0 for |t| < 2^-5 (the
//                    series converges for |t| < sqrt(nu)); above, |t| =
//                    2^E m, m in [1, 2), is split by its exponent and the top
//                    5 bits of m into segments of relative width 1/32, and
//                    each row holds G as a series in r = m / m_c - 1 about
//                    the segment centre m_c: the ODE in y = log t,
//                    (nu + e^{2y}) G_yy = nu (1 - e^{2y}) G_y + (nu + e^{2y}) G G_y^2,
//                    gives G's series in y, composed with y = y_c + log(1 + r).
//                    The device thus needs no logarithm: exponent and mantissa
//                    bits select the row, one FMA forms r.
//
// Each segment's expansion is computed at its centre c from the value and the
// slope there (Q(c) by inverting the special function in long double, Q'(c)
// = f_0 / f_1), the higher Taylor coefficients by the ODE's recurrence, so
// there is no integration and no error growth in either tail; every segment
// is checked against direct values at both of its ends.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>
#include <vector>

#include "qm.h"
#include "qm_host.h"
#include "qm_t_fx.h"

namespace qm {
namespace {

using LD = long double;
constexpr LD kPi = 3.14159265358979323846264338327950288L;
constexpr LD kLnSqrt2Pi = 0.91893853320467274178032973640561764L;
constexpr LD kLn2 = 0.69314718055994530941723212145817657L;
constexpr int DI = 18;   // working degree of the local series
constexpr int DO = 9;    // stored degree
constexpr int RW = 11;   // doubles per row: DO + 1 coefficients, then the centre
                         // (log W rows) or 1 / m_c (G rows)

// ---- special functions, long double -------------------------------------

// log of Phi(z) and of 1 - Phi(z)
LD log_ncdf(LD z) { return std::log(0.5L * std::erfc(-z / std::sqrt(2.0L))); }
LD log_nsf(LD z) { return std::log(0.5L * std::erfc(z / std::sqrt(2.0L))); }

// log P(a, e^lx) by the power series of the lower incomplete gamma function
LD log_p_series(LD a, LD lx)
{
    const LD x = std::exp(lx);
    LD t = 1.0L, sum = 1.0L;
    for (int n = 1; n < 200000 && t > 1e-22L * sum; ++n) {
        t *= x / (a + n);
        sum += t;
    }
    return a * lx - x - std::lgamma(a + 1.0L) + std::log(sum);
}

// log Q(a, e^lx) by Legendre's continued fraction of the upper function,
// evaluated with the modified Lentz recurrence
LD log_q_fraction(LD a, LD lx)
{
    const LD x = std::exp(lx), tiny = 1e-4000L;
    LD bn = x + 1.0L - a, c = 1.0L / tiny, d = 1.0L / bn, h = d;
    for (int n = 1; n < 200000; ++n) {
        const LD an = n * (a - n);
        bn += 2.0L;
        d = bn + an * d;
        c = bn + an / c;
        if (std::fabs(d) < tiny) d = tiny;
        if (std::fabs(c) < tiny) c = tiny;
        d = 1.0L / d;
        const LD f = c * d;
        h *= f;
        if (std::fabs(f - 1.0L) < 1e-21L) break;
    }
    return a * lx - x - std::lgamma(a) + std::log(h);
}

LD log_gp(LD a, LD lx) { return std::exp(lx) < a + 1 ? log_p_series(a, lx) : std::log1p(-std::exp(log_q_fraction(a, lx))); }
LD log_gq(LD a, LD lx) { return std::exp(lx) < a + 1 ? std::log1p(-std::exp(log_p_series(a, lx))) : log_q_fraction(a, lx); }

// s = log(W/2) with P(W <= w) = Phi(z), W ~ chi-squared(2a)
LD chi2_log_half(LD a, LD z)
{
    const bool lower = z <= 0;
    const LD target = lower ? log_ncdf(z) : log_nsf(z);
    LD lo = -20000.0L, hi = 30.0L;
    LD s = lower ? (target + std::lgamma(a + 1.0L)) / a : std::log(a + z * z + 2 * z * std::sqrt(a) + 1);
    if (!(s > lo && s < hi)) s = 0.5L * (lo + hi);
    for (int it = 0; it < 500; ++it) {
        const LD lp = lower ? log_gp(a, s) : log_gq(a, s);
        const LD g = lower ? lp - target : target - lp;           // increasing in s
        if (g == 0) break;
        (g > 0 ? hi : lo) = s;
        const LD slope = std::exp(a * s - std::exp(s) - std::lgamma(a) - lp);
        LD sn = s - g / slope;
        if (!(sn > lo && sn < hi)) sn = 0.5L * (lo + hi);
        const bool done = std::fabs(sn - s) <= 1e-19L * std::fmax(1.0L, std::fabs(s));
        s = sn;
        if (done) break;
    }
    return s;
}

// I_x(a, b) by the continued fraction of DLMF 8.17.22 (x below its mean
// (a+1)/(a+b+2)); returns log I_x
LD log_ibeta_cf(LD a, LD b, LD x)
{
    const LD tiny = 1e-4000L;
    LD c = 1.0L, d = 1.0L - (a + b) * x / (a + 1.0L);
    if (std::fabs(d) < tiny) d = tiny;
    d = 1.0L / d;
    LD h = d;
    for (int m = 1; m < 200000; ++m) {
        const LD m2 = 2.0L * m;
        LD num = m * (b - m) * x / ((a + m2 - 1) * (a + m2));
        d = 1.0L + num * d;
        c = 1.0L + num / c;
        if (std::fabs(d) < tiny) d = tiny;
        if (std::fabs(c) < tiny) c = tiny;
        d = 1.0L / d;
        h *= d * c;
        num = -(a + m) * (a + b + m) * x / ((a + m2) * (a + m2 + 1));
        d = 1.0L + num * d;
        c = 1.0L + num / c;
        if (std::fabs(d) < tiny) d = tiny;
        if (std::fabs(c) < tiny) c = tiny;
        d = 1.0L / d;
        const LD f = d * c;
        h *= f;
        if (std::fabs(f - 1.0L) < 1e-21L) break;
    }
    const LD lbeta = std::lgamma(a) + std::lgamma(b) - std::lgamma(a + b);
    return a * std::log(x) + b * std::log1p(-x) - lbeta - std::log(a) + std::log(h);
}

// g >= 0 with log(1 - Phi(g)) = lp (tail form), or erf(g/sqrt2) = q (centre)
LD probit_tail_log(LD lp)
{
    LD g = std::sqrt(std::fmax(-2 * lp - std::log(-4 * kPi * lp), 0.25L)), lo = 0.0L, hi = 40.0L;
    for (int it = 0; it < 300; ++it) {
        const LD f = log_nsf(g) - lp;                                  // decreasing in g
        (f > 0 ? lo : hi) = g;
        const LD dl = -std::exp(-g * g / 2 - kLnSqrt2Pi - log_nsf(g));   // d/dg log(1 - Phi)
        LD gn = g - f / dl;
        if (!(gn > lo && gn < hi)) gn = 0.5L * (lo + hi);
        const bool done = std::fabs(gn - g) <= 1e-20L * std::fmax(1.0L, g);
        g = gn;
        if (done) break;
    }
    return g;
}

LD probit_centre(LD q)
{
    LD g = 1.2533141373155002512L * q, lo = 0.0L, hi = 12.0L;   // sqrt(pi/2) q
    for (int it = 0; it < 300; ++it) {
        const LD f = std::erf(g / std::sqrt(2.0L)) - q;
        (f > 0 ? hi : lo) = g;
        const LD df = 2.0L * std::exp(-g * g / 2 - kLnSqrt2Pi);
        LD gn = g - f / df;
        if (!(gn > lo && gn < hi)) gn = 0.5L * (lo + hi);
        const bool done = std::fabs(gn - g) <= 1e-20L * std::fmax(1e-300L, g);
        g = gn;
        if (done) break;
    }
    return g;
}

// G(t) = Phi^{-1}(F_nu(t)) for t > 0
LD t_to_normal(LD nu, LD t)
{
    const LD a = nu / 2;
    const LD x = nu / (nu + t * t);                      // P(T > t) = I_x(a, 1/2) / 2
    if (x < (a + 1) / (a + 2.5L)) {                     // below the mean of I_x(a, 1/2)
        const LD lp = log_ibeta_cf(a, 0.5L, x) - kLn2;
        if (lp < std::log(0.25L)) return probit_tail_log(lp);
        return probit_centre(-std::expm1(lp + kLn2));    // 2 F(t) - 1 = 1 - 2p
    }
    const LD y = t * t / (nu + t * t);                   // 2 F(t) - 1 = I_y(1/2, a)
    return probit_centre(std::exp(log_ibeta_cf(0.5L, a, y)));
}

// ---- series ---------------------------------------------------------------

using Ser = std::vector<LD>;

Ser smul(const Ser& p, const Ser& q)
{
    Ser r(p.size(), 0.0L);
    for (size_t i = 0; i < p.size(); ++i)
        for (size_t k = 0; i + k < p.size(); ++k) r[i + k] += p[i] * q[k];
    return r;
}

Ser sderiv(const Ser& p)
{
    Ser r(p.size(), 0.0L);
    for (size_t k = 0; k + 1 < p.size(); ++k) r[k] = (k + 1) * p[k + 1];
    return r;
}

// W W'' = -(c+s) W W' - (k-1) W'^2 + W W'^2 / 2, W(c) = w0, W'(c) = w1
Ser taylor_chi2(LD k, LD c, LD w0, LD w1)
{
    Ser b(DI + 1, 0.0L);
    b[0] = w0;
    b[1] = w1;
    for (int n = 0; n + 2 <= DI; ++n) {
        const Ser d1 = sderiv(b);
        Ser d2 = sderiv(d1);
        d2[n] = 0.0L;                                   // (m+2)(m+1) b_{m+2}, m = n unknown
        const Ser P = smul(b, d1), Q2 = smul(d1, d1), R = smul(b, Q2), WW = smul(b, d2);
        const LD rhs = -c * P[n] - (n >= 1 ? P[n - 1] : 0.0L) - (k - 1) * Q2[n] + 0.5L * R[n];
        b[n + 2] = (rhs - WW[n]) / (b[0] * (n + 2) * (n + 1));
    }
    return b;
}

// log of a series with b_0 > 0
Ser slog(const Ser& b)
{
    Ser f(b.size(), 0.0L), a(b.size(), 0.0L);
    for (size_t k = 1; k < b.size(); ++k) a[k] = b[k] / b[0];
    f[0] = std::log(b[0]);
    for (size_t k = 1; k < b.size(); ++k) {             // (1 + a) f' = a'
        LD acc = k * a[k];
        for (size_t i = 1; i < k; ++i) acc -= a[i] * (k - i) * f[k - i];
        f[k] = acc / k;
    }
    return f;
}

// (nu + t^2) G'' = -(nu+1) t G' + (nu + t^2) G G'^2 about t = c
Ser taylor_g_t(LD nu, LD c, LD g0, LD g1)
{
    Ser b(DI + 1, 0.0L), A(DI + 1, 0.0L), T(DI + 1, 0.0L);
    A[0] = nu + c * c;
    A[1] = 2 * c;
    A[2] = 1.0L;
    T[0] = c;
    T[1] = 1.0L;
    b[0] = g0;
    b[1] = g1;
    for (int n = 0; n + 2 <= DI; ++n) {
        const Ser d1 = sderiv(b);
        Ser d2 = sderiv(d1);
        d2[n] = 0.0L;
        const Ser Ad2 = smul(A, d2), Td1 = smul(T, d1), GQ = smul(b, smul(d1, d1)), AGQ = smul(A, GQ);
        const LD rhs = -(nu + 1) * Td1[n] + AGQ[n];
        b[n + 2] = (rhs - Ad2[n]) / (A[0] * (n + 2) * (n + 1));
    }
    return b;
}

// in y = log t about y = c: dividing the ODE by e^{2c},
// (nu e^{-2c} + e^{2s}) G'' = nu (e^{-2c} - e^{2s}) G' + (nu e^{-2c} + e^{2s}) G G'^2
Ser taylor_g_y(LD nu, LD c, LD g0, LD g1)
{
    Ser b(DI + 1, 0.0L), E(DI + 1, 0.0L), B(DI + 1, 0.0L), C(DI + 1, 0.0L);
    const LD em = nu * std::exp(-2 * c);
    LD f = 1.0L;
    for (int m = 0; m <= DI; ++m) {
        E[m] = f;                                       // e^{2s} = sum (2s)^m / m!
        f *= 2.0L / (m + 1);
    }
    for (int m = 0; m <= DI; ++m) {
        B[m] = E[m] + (m == 0 ? em : 0.0L);
        C[m] = -nu * E[m] + (m == 0 ? em : 0.0L);
    }
    b[0] = g0;
    b[1] = g1;
    for (int n = 0; n + 2 <= DI; ++n) {
        const Ser d1 = sderiv(b);
        Ser d2 = sderiv(d1);
        d2[n] = 0.0L;
        const Ser Bd2 = smul(B, d2), Cd1 = smul(C, d1), BGQ = smul(B, smul(b, smul(d1, d1)));
        const LD rhs = Cd1[n] + BGQ[n];
        b[n + 2] = (rhs - Bd2[n]) / (B[0] * (n + 2) * (n + 1));
    }
    return b;
}

// G's series in r from its series in y about y_c: y - y_c = log(1 + r)
Ser compose_log1p(const Ser& gy)
{
    Ser L(DI + 1, 0.0L), P(DI + 1, 0.0L), out(DI + 1, 0.0L);
    for (int k = 1; k <= DI; ++k) L[k] = ((k & 1) ? 1.0L : -1.0L) / k;     // log(1 + r)
    P[0] = 1.0L;                                                           // L^0
    for (int k = 0; k <= DI; ++k) {
        for (int i = 0; i <= DI; ++i) out[i] += gy[k] * P[i];
        P = smul(P, L);
    }
    return out;
}

LD hornerl(const Ser& b, int D, LD s)
{
    LD r = b[D];
    for (int k = D - 1; k >= 0; --k) r = r * s + b[k];
    return r;
}

}  // namespace

// Tables for nu in host memory (layout in qm.h, qm_tcopula_table_build).
qm_status tcop_table_build(double nu_d, double* chi_seg, double* g_seg, int* ne_out)
{
    if (!(nu_d >= QM_T_NU_MIN && nu_d <= QM_T_NU_MAX))
        return fail(QM_ERR_UNSUPPORTED, "t copula: nu = %g outside [%g, %g]", nu_d, QM_T_NU_MIN, QM_T_NU_MAX);
    const LD nu = nu_d, k = nu / 2;
    const LD lgk = std::lgamma(k);

    // ---- mixing variable: L = log W on z in [-Z, Z], width 1/16 ----------
    const LD hz = 1.0L / QM_TC_HZ_INV;
    auto logw = [&](LD z) { return kLn2 + chi2_log_half(k, z); };
    LD worst = 0.0L;
    for (int j = 0; j < QM_TC_NZ; ++j) {
        const LD c = -(LD)QM_TC_Z_MAX + (j + 0.5L) * hz;
        const LD lw = logw(c), w0 = std::exp(lw);
        // W' = phi(c) / f(W), log f(w) = (k-1) log w - w/2 - k ln 2 - lgamma(k)
        const LD lf = (k - 1) * lw - w0 / 2 - k * kLn2 - lgk;
        const LD w1 = std::exp(-c * c / 2 - kLnSqrt2Pi - lf);
        const Ser L = slog(taylor_chi2(k, c, w0, w1));
        if (!std::isfinite(L[DI]))
            return fail(QM_ERR_INVALID, "t copula: chi-squared series overflow for nu = %g", nu_d);
        for (int e = -1; e <= 1; e += 2) {
            const LD err = std::fabs(hornerl(L, DO, e * hz / 2) - logw(c + e * hz / 2));
            worst = std::fmax(worst, err);
        }
        for (int q = 0; q <= DO; ++q) chi_seg[RW * j + q] = (double)L[q];
        chi_seg[RW * j + DO + 1] = (double)c;
    }
    if (!(worst < 1e-13L))
        return fail(QM_ERR_INVALID, "t copula: chi-squared table check failed for nu = %g (%Lg)", nu_d, worst);

    // largest |T| the sampler can produce: |y_j| / sigma_j <= |eps| <= 8.3 sqrt(16)
    // times S = sqrt(nu / W) at the smallest grid normal
    const LD smax = std::exp(0.5L * (std::log(nu) - logw(-8.3L)));
    const int emax = (int)std::floor(std::log2(8.3L * 4.0L * smax)) + 1;        // last binade, inclusive
    const int ne = emax - QM_TC_G_EMIN + 1;
    if (ne > QM_TC_G_NE_MAX)
        return fail(QM_ERR_UNSUPPORTED, "t copula: nu = %g needs %d binades (max %d)", nu_d, ne, QM_TC_G_NE_MAX);

    // ---- t -> normal: row 0 about t = 0, then 32 segments per binade -------
    const LD lft0 = std::lgamma((nu + 1) / 2) - lgk - 0.5L * std::log(nu * kPi);   // log f_nu(0)
    auto logft = [&](LD t) { return lft0 - (nu + 1) / 2 * std::log1p(t * t / nu); };
    const int nseg = 1 << QM_TC_G_K;
    worst = 0.0L;
    {
        const Ser b = taylor_g_t(nu, 0.0L, 0.0L, std::exp(lft0 + kLnSqrt2Pi));  // G'(0) = f_nu(0) / phi(0)
        for (LD t : {std::ldexp(1.0L, QM_TC_G_EMIN), std::ldexp(0.75L, QM_TC_G_EMIN), 1e-3L})
            worst = std::fmax(worst, std::fabs(hornerl(b, DO, t) / t_to_normal(nu, t) - 1));
        for (int q = 0; q <= DO; ++q) g_seg[q] = (double)b[q];
        g_seg[DO + 1] = 0.0;
    }
    for (int e = 0; e < ne; ++e) {
        const int E = QM_TC_G_EMIN + e;
        for (int j = 0; j < nseg; ++j) {
            const LD mc = 1.0L + (j + 0.5L) / nseg;
            const LD yc = E * kLn2 + std::log(mc);
            const LD t = std::exp(yc), g0 = t_to_normal(nu, t);
            const LD g1 = t * std::exp(logft(t) + g0 * g0 / 2 + kLnSqrt2Pi);         // dG/dy = t G'
            const Ser b = compose_log1p(taylor_g_y(nu, yc, g0, g1));
            if (!std::isfinite(b[DI]))
                return fail(QM_ERR_INVALID, "t copula: t -> normal series overflow for nu = %g", nu_d);
            for (LD m : {1.0L + (LD)j / nseg, 1.0L + (j + 1.0L) / nseg}) {
                const LD ref = t_to_normal(nu, std::ldexp(m, E));
                worst = std::fmax(worst, std::fabs(hornerl(b, DO, m / mc - 1) / ref - 1));
            }
            double* row = g_seg + RW * (1 + e * nseg + j);
            for (int q = 0; q <= DO; ++q) row[q] = (double)b[q];
            row[DO + 1] = (double)(1.0L / mc);
        }
    }
    if (!(worst < 1e-13L))
        return fail(QM_ERR_INVALID, "t copula: t -> normal table check failed for nu = %g (%Lg)", nu_d, worst);
    *ne_out = ne;
    return QM_OK;
}

namespace {

// Device row: coefficients 0..4 in double, 5..9 in single precision (their
// rounding stays below 2e-15 relative on every row), the layout of the
// Student-t segments, so the same mixed evaluation serves both.
struct PackedRow {
    double a[5];
    float b[5];
    float pad;
};
static_assert(sizeof(PackedRow) == 64, "packed row layout");

struct TcEntry {
    int device;
    double nu;
    void* chi;     // device: QM_TC_NZ packed rows, then QM_TC_NZ centres
    void* g;       // device: 1 + ne 2^QM_TC_G_K packed rows, then as many 1 / m_c
    void* fx;      // device: QM_TC_NZ fixed-point log W rows, then 1 + ne 2^QM_TC_G_K G rows
    int ne;
};

// The fixed-point rows (pack_fx_biased): log W on [j/16 - z_max, + 1/16)
// about its centre; G row 0 the series about t = 0 on [0, 2^G_EMIN); G row
// 1 + e 2^K + j on |t| in [2^E (1 + j/32), + 2^(E-5)), E = G_EMIN + e, its
// series in r = m / m_c - 1 turned into one in s = |t| - 2^E m_c
// (coefficient k divided by (2^E m_c)^k).
qm_status tcop_pack_fx(const double* hc, const double* hg, int ne, std::vector<ttbl::SegTX>& fx)
{
    const int ng = 1 + ne * (1 << QM_TC_G_K);
    fx.assign(QM_TC_NZ + ng, ttbl::SegTX{});
    const double wz = 1.0 / QM_TC_HZ_INV;
    for (int j = 0; j < QM_TC_NZ; ++j) {
        const double start = j * wz - QM_TC_Z_MAX;
        const qm_status st = pack_fx_biased(&hc[RW * j], wz, hc[RW * j + DO + 1] - start, &fx[j]);
        if (st != QM_OK) return st;
    }
    qm_status st = pack_fx_biased(&hg[0], std::ldexp(1.0, QM_TC_G_EMIN), 0.0, &fx[QM_TC_NZ]);
    if (st != QM_OK) return st;
    for (int i = 1; i < ng; ++i) {
        const int E = QM_TC_G_EMIN + ((i - 1) >> QM_TC_G_K);
        const double cabs = std::ldexp(1.0, E) / hg[RW * i + DO + 1];
        double b[DO + 1];
        double p = 1.0;
        for (int k = 0; k <= DO; ++k) {
            b[k] = hg[RW * i + k] / p;
            p *= cabs;
        }
        st = pack_fx_biased(b, std::ldexp(1.0, E - QM_TC_G_K), std::ldexp(1.0, E - QM_TC_G_K - 1), &fx[QM_TC_NZ + i]);
        if (st != QM_OK) return st;
    }
    return QM_OK;
}

std::mutex g_tc_mu;
std::vector<TcEntry> g_tc_cache;
constexpr size_t kTcMax = 256;

// host rows of RW doubles -> packed rows followed by the rows' last values
std::vector<unsigned char> pack_rows(const double* rows, int n)
{
    std::vector<unsigned char> buf((sizeof(PackedRow) + sizeof(double)) * (size_t)n);
    PackedRow* pr = reinterpret_cast<PackedRow*>(buf.data());
    double* last = reinterpret_cast<double*>(buf.data() + sizeof(PackedRow) * (size_t)n);
    for (int i = 0; i < n; ++i) {
        const double* r = rows + (size_t)RW * i;
        for (int k = 0; k < 5; ++k) pr[i].a[k] = r[k];
        for (int k = 0; k < 5; ++k) pr[i].b[k] = (float)r[5 + k];
        pr[i].pad = 0.0f;
        last[i] = r[DO + 1];
    }
    return buf;
}

}  // namespace

// Device tables for nu on the current device, built and uploaded at first use
// (kept until the process exits): packed rows, then the rows' centres (log W)
// or 1 / m_c (G).
qm_status tcop_table_device(double nu, const void** chi, const void** g, const void** fx, int* ne)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail(QM_ERR_CUDA, "t copula: no current device");
    std::lock_guard<std::mutex> lk(g_tc_mu);
    for (const TcEntry& e : g_tc_cache)
        if (e.device == dev && e.nu == nu) {
            *chi = e.chi;
            *g = e.g;
            *fx = e.fx;
            *ne = e.ne;
            return QM_OK;
        }
    if (g_tc_cache.size() >= kTcMax) return fail(QM_ERR_NOMEM, "t copula: more than %zu distinct nu in use", kTcMax);
    std::vector<double> hc(RW * QM_TC_NZ), hg(RW * (1 + QM_TC_G_NE_MAX * (1 << QM_TC_G_K)));
    int n = 0;
    const qm_status st = tcop_table_build(nu, hc.data(), hg.data(), &n);
    if (st != QM_OK) return st;
    const std::vector<unsigned char> pc = pack_rows(hc.data(), QM_TC_NZ);
    const std::vector<unsigned char> pg = pack_rows(hg.data(), 1 + n * (1 << QM_TC_G_K));
    std::vector<ttbl::SegTX> pf;
    const qm_status pst = tcop_pack_fx(hc.data(), hg.data(), n, pf);
    if (pst != QM_OK) return pst;
    const size_t fbytes = sizeof(ttbl::SegTX) * pf.size();
    TcEntry e{dev, nu, nullptr, nullptr, nullptr, n};
    if (cudaMalloc(&e.chi, pc.size()) != cudaSuccess || cudaMalloc(&e.g, pg.size()) != cudaSuccess ||
        cudaMalloc(&e.fx, fbytes) != cudaSuccess) {
        if (e.chi) cudaFree(e.chi);
        if (e.g) cudaFree(e.g);
        return fail(QM_ERR_NOMEM, "t copula: table allocation failed");
    }
    if (cudaMemcpy(e.chi, pc.data(), pc.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(e.g, pg.data(), pg.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(e.fx, pf.data(), fbytes, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(e.chi);
        cudaFree(e.g);
        cudaFree(e.fx);
        return fail(QM_ERR_CUDA, "t copula: table upload failed");
    }
    g_tc_cache.push_back(e);
    *chi = e.chi;
    *g = e.g;
    *fx = e.fx;
    *ne = e.ne;
    return QM_OK;
}

}  // namespace qm

extern "C" qm_status qm_tcopula_table_build(double nu, double* chi_seg, double* g_seg, int* ne)
{
    if (!chi_seg || !g_seg || !ne) return qm::fail(QM_ERR_INVALID, "qm_tcopula_table_build: null argument");
    return qm::tcop_table_build(nu, chi_seg, g_seg, ne);
}
