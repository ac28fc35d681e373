// qm_tdyn.cu -- normal -> Student t recycling tables for any real nu, built
// on the host at first use (Sec. 3).
//
// The map Q(z) = F_nu^{-1}(Phi(z)) satisfies the Gaussian-background
// recycling ODE (Sec. 3.1)
//     (1 + Q^2/nu)(Q'' + z Q') = (1 + 1/nu) Q Q'^2 .
// Matching powers of s in Q(z0 + s) = sum_k b_k s^k gives b_{k+2} from
// b_0..b_{k+1} (the recurrence of Sec. 3.2, taken at any expansion point
// z0).  The table holds, for the segments [j/32, (j+1)/32) of 0 <= z < 8.75,
// the local expansion about the segment centre (about 0 for j = 0, where it
// is the paper's central series with Q'(0) = gamma).
//
// Q and Q' at the centres come from integrating the ODE with these series,
// BACKWARDS from the tail: a perturbation of Q grows like 1/(1 - Phi(z))
// when integrating towards larger z (forward integration from z = 0 loses
// all accuracy by z ~ 8), and decays in the other direction.  The start
// values come from the tail coordinate of Sec. 3.3,
//     w = kappa (1 - Phi(z)),  kappa = nu B(nu/2, 1/2),
//     Q = sqrt(nu) w^{-1/nu} R(y),  y = w^{2/nu},
// whose power series R(y) (R(0) = 1, R'(0) = -(nu+1)/(2(nu+2))) is obtained
// here by series reversion of the exact tail of the Student distribution,
//     P(T > t) = I_x(nu/2, 1/2)/2 = x^{nu/2} (1-x)^{1/2} 2F1((nu+1)/2, 1; nu/2+1; x)/(nu B),
//     x = nu/(nu + t^2) = s/(1+s),  s = nu/t^2,
// so that y = s g(s) with g = (1+s)^{-(1+1/nu)} 2F1(...)^{2/nu}, s(y) by
// reversion and R = (y/s)^{1/2}.  The device uses the same series for
// z >= 8.75.  Everything here is long double; the integration's consistency
// with the central series (Q(0) = 0, Q'(0) = gamma) is checked.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <mutex>
#include <vector>

#include "qm.h"
#include "qm_host.h"
#include "qm_t_fx.h"
#include "qm_t_tables.h"

namespace qm {
namespace {

using LD = long double;
constexpr int NSEG = ttbl::NSEG;     // 280 segments of width 1/32
constexpr int H_INV = ttbl::H_INV;
constexpr int DEG_INT = 22;          // series degree used for the integration
constexpr int NT = QM_T_TAIL_TERMS;  // tail series terms R_0..R_{NT-1}
constexpr int NS = NT + 2;           // working length of the series (the reversion
                                     // below loses the last term of s/y)

using Ser = std::vector<LD>;

Ser ser_mul(const Ser& a, const Ser& b)
{
    Ser c(NS, 0.0L);
    for (int i = 0; i < NS; ++i)
        for (int k = 0; i + k < NS; ++k) c[i + k] += a[i] * b[k];
    return c;
}

// log(1 + a) for a series with a[0] = 0: k f_k = k a_k - sum_{i=1}^{k-1} a_i (k-i) f_{k-i}
Ser ser_log1p(const Ser& a)
{
    Ser f(NS, 0.0L);
    for (int k = 1; k < NS; ++k) {
        LD acc = k * a[k];
        for (int i = 1; i < k; ++i) acc -= a[i] * (k - i) * f[k - i];
        f[k] = acc / k;
    }
    return f;
}

// exp(a) for a series with a[0] = 0: k e_k = sum_{i=1}^{k} i a_i e_{k-i}
Ser ser_exp(const Ser& a)
{
    Ser e(NS, 0.0L);
    e[0] = 1.0L;
    for (int k = 1; k < NS; ++k) {
        LD acc = 0.0L;
        for (int i = 1; i <= k; ++i) acc += i * a[i] * e[k - i];
        e[k] = acc / k;
    }
    return e;
}

// R_0..R_{NS-1} of the tail coordinate (see the file comment)
Ser tail_series(LD nu)
{
    Ser s1(NS, 0.0L);
    s1[1] = 1.0L;                                   // the series "s"
    Ser x(NS, 0.0L);                                // x = s/(1+s)
    for (int k = 1; k < NS; ++k) x[k] = (k % 2) ? 1.0L : -1.0L;
    const LD a = (nu + 1) / 2, c = nu / 2 + 1;
    Ser F1(NS, 0.0L), p(NS, 0.0L);
    p[0] = 1.0L;
    LD coef = 1.0L;
    for (int k = 1; k < NS; ++k) {                  // 2F1(a, 1; c; x) - 1
        p = ser_mul(p, x);
        coef *= (a + k - 1) / (c + k - 1);
        for (int i = 0; i < NS; ++i) F1[i] += coef * p[i];
    }
    const Ser l1s = ser_log1p(s1), lF = ser_log1p(F1);
    Ser lg(NS), mlg(NS);
    for (int k = 0; k < NS; ++k) {
        lg[k] = -(1 + 1 / nu) * l1s[k] + (2 / nu) * lF[k];
        mlg[k] = -lg[k];
    }
    const Ser ginv = ser_exp(mlg);                  // 1/g(s)
    // reversion of y = s g(s): s = y / g(s), iterated (each pass fixes one more term)
    Ser s(NS, 0.0L);
    s[1] = 1.0L;
    for (int it = 0; it < NS; ++it) {
        Ser comp(NS, 0.0L);
        comp[0] = ginv[NS - 1];
        for (int k = NS - 2; k >= 0; --k) {         // Horner in series arithmetic
            comp = ser_mul(comp, s);
            comp[0] += ginv[k];
        }
        for (int k = NS - 1; k >= 1; --k) s[k] = comp[k - 1];
        s[0] = 0.0L;
    }
    // R = (s/y)^{-1/2}, s/y = s[1] + s[2] y + ...
    Ser sy(NS, 0.0L);
    for (int k = 0; k + 1 < NS; ++k) sy[k] = s[k + 1];
    Ser d(NS, 0.0L);
    for (int k = 1; k < NS; ++k) d[k] = sy[k];      // sy[0] = 1
    Ser lr = ser_log1p(d);
    for (auto& v : lr) v *= -0.5L;
    return ser_exp(lr);
}

// b_0..b_D of Q(z0 + s) for the Gaussian-background Student-t ODE
void taylor_at(LD nu, LD z0, LD q0, LD q1, int D, LD* b)
{
    b[0] = q0;
    b[1] = q1;
    std::vector<LD> A(D + 1), d1(D + 1), q2(D + 1), d1sq(D + 1), L(D + 1);
    for (int n = 0; n + 2 <= D; ++n) {
        // series up to index n with b_{n+2} still unknown
        for (int i = 0; i <= n; ++i) {
            LD acc = 0.0L;
            for (int j = 0; j <= i; ++j) acc += b[j] * b[i - j];
            q2[i] = acc;
            A[i] = (i == 0 ? 1.0L : 0.0L) + acc / nu;
            d1[i] = (i + 1) * b[i + 1];
        }
        for (int i = 0; i <= n; ++i) {
            LD acc = 0.0L;
            for (int j = 0; j <= i; ++j) acc += d1[j] * d1[i - j];
            d1sq[i] = acc;
        }
        // L_m = (m+2)(m+1) b_{m+2} + z0 (m+1) b_{m+1} + m b_m, known for m < n
        for (int m = 0; m < n; ++m) L[m] = (m + 2) * (m + 1) * b[m + 2] + z0 * (m + 1) * b[m + 1] + m * b[m];
        LD lhs = A[0] * (z0 * (n + 1) * b[n + 1] + n * b[n]);
        for (int i = 1; i <= n; ++i) lhs += A[i] * L[n - i];
        LD rhs = 0.0L;
        for (int i = 0; i <= n; ++i) rhs += b[i] * d1sq[n - i];
        rhs *= (1 + 1 / nu);
        b[n + 2] = (rhs - lhs) / (A[0] * (n + 2) * (n + 1));
    }
}

LD horner(const LD* b, int D, LD s)
{
    LD r = b[D];
    for (int k = D - 1; k >= 0; --k) r = r * s + b[k];
    return r;
}

LD horner_d(const LD* b, int D, LD s)
{
    LD r = D * b[D];
    for (int k = D - 1; k >= 1; --k) r = r * s + k * b[k];
    return r;
}

}  // namespace

// Builds the tables for nu (host memory).  seg: NSEG x 10 coefficients
// (coefficient k of segment j at seg[10 j + k]); tail: nu, log kappa, degree,
// R_0..R_degree.  Returns QM_OK or an error with a message.
qm_status t_table_build(double nu_d, double* seg, double* tail)
{
    if (!(nu_d >= QM_T_NU_MIN && nu_d <= QM_T_NU_MAX))
        return fail(QM_ERR_UNSUPPORTED, "Student t: nu = %g outside [%g, %g]", nu_d, QM_T_NU_MIN,
                    QM_T_NU_MAX);
    const LD nu = nu_d;
    const LD lB = std::lgamma(nu / 2) + 0.5L * std::log(3.14159265358979323846264338327950288L) -
                  std::lgamma((nu + 1) / 2);                               // log B(nu/2, 1/2)
    const LD log_kappa = std::log(nu) + lB;
    const LD gamma = std::sqrt(nu / 2) * std::exp(std::lgamma(nu / 2) - std::lgamma((nu + 1) / 2));
    const Ser R = tail_series(nu);
    const LD r1 = -(nu + 1) / (2 * (nu + 2));
    if (std::fabs(R[1] - r1) > 1e-15L * std::fabs(r1))
        return fail(QM_ERR_INVALID, "Student t: tail series check failed for nu = %g", nu_d);

    // start on the grid z = (2J+1)/64 at the last segment centre, further out
    // until y <= 0.1 (the tail series then converges to far below 1e-15)
    const LD ln_sqrt2pi = 0.91893853320467274178032973640561764L;
    auto log_upper = [](LD z) { return std::log(0.5L * std::erfc(z / std::sqrt(2.0L))); };
    long J = NSEG - 1;                                       // centre (2J+1)/64
    LD z = (2 * J + 1) / (LD)(2 * H_INV), lw = log_kappa + log_upper(z);
    while (std::exp(2 * lw / nu) > 0.1L && J < NSEG + 64 * H_INV) {
        ++J;
        z = (2 * J + 1) / (LD)(2 * H_INV);
        lw = log_kappa + log_upper(z);
    }
    {
        const LD y = std::exp(2 * lw / nu);
        LD Ry = 0.0L, dRy = 0.0L;
        for (int k = NT - 1; k >= 0; --k) Ry = Ry * y + R[k];
        for (int k = NT - 1; k >= 1; --k) dRy = dRy * y + k * R[k];
        // Q = sqrt(nu) w^{-1/nu} R(y); Q' = kappa phi(z) w^{-1/nu-1} (R - 2 y R') / sqrt(nu)
        const LD q = std::sqrt(nu) * std::exp(-lw / nu) * Ry;
        const LD lqp = log_kappa - z * z / 2 - ln_sqrt2pi - (1 / nu + 1) * lw +
                       std::log(Ry - 2 * y * dRy) - 0.5L * std::log(nu);
        LD qp = std::exp(lqp);
        LD b[DEG_INT + 1];
        LD qc = q;
        const LD h = 1.0L / H_INV;
        for (; J >= 1; --J) {
            z = (2 * J + 1) / (LD)(2 * H_INV);
            taylor_at(nu, z, qc, qp, DEG_INT, b);
            if (!std::isfinite(b[DEG_INT]))
                return fail(QM_ERR_INVALID, "Student t: integration overflow for nu = %g", nu_d);
            if (J < NSEG)
                for (int k = 0; k < 10; ++k) seg[10 * J + k] = (double)b[k];
            if (J == 1) break;
            qc = horner(b, DEG_INT, -h);
            qp = horner_d(b, DEG_INT, -h);
        }
        // segment 0: the central series (Sec. 3.2), Q(0) = 0, Q'(0) = gamma;
        // it must agree with the integrated solution at the centre of segment 1
        LD c[DEG_INT + 1];
        taylor_at(nu, 0.0L, 0.0L, gamma, DEG_INT, c);
        for (int k = 0; k < 10; ++k) seg[k] = (double)c[k];
        const LD z1 = 3.0L / (2 * H_INV);
        const LD qcen = horner(c, DEG_INT, z1);
        if (std::fabs(qcen / b[0] - 1) > 1e-13L)
            return fail(QM_ERR_INVALID, "Student t: integration inconsistent with the central series "
                        "for nu = %g (%Lg)", nu_d, qcen / b[0] - 1);
    }
    tail[0] = nu_d;
    tail[1] = (double)log_kappa;
    tail[2] = NT - 1;
    for (int k = 0; k < NT; ++k) tail[3 + k] = (double)R[k];
    return QM_OK;
}

// Segment rows in the fixed-point form of qm_t_fx.h (280 rows per nu).  The
// re-expansion is done in double: its k = m term dominates every sum, so the
// rounding stays at a few ulp, far inside the map's 1e-12 bound (and long
// double is a software quad type on some hosts, slow at first use).
static_assert(ttbl::T_NROW == QM_T_NROW && sizeof(ttbl::TRows) == QM_T_ROWS_BYTES,
              "the row layout qm.h documents");

qm_status t_pack_rows(const double* seg10, int nseg, ttbl::TRows* out)
{
    // double precision throughout: the conversion runs at the first use of a
    // table on a device (for the offline tables inside the first Student-t
    // call), and long double is software-emulated on some hosts (128-bit on
    // aarch64), which made that first call take tens of milliseconds
    using LD = double;
    static const LD binom[10][10] = {
        {1}, {1, 1}, {1, 2, 1}, {1, 3, 3, 1}, {1, 4, 6, 4, 1}, {1, 5, 10, 10, 5, 1},
        {1, 6, 15, 20, 15, 6, 1}, {1, 7, 21, 35, 35, 21, 7, 1}, {1, 8, 28, 56, 70, 56, 28, 8, 1},
        {1, 9, 36, 84, 126, 126, 84, 36, 9, 1}};
    constexpr int DIV = ttbl::T_ROWS_PER_UNIT / H_INV;             // rows per segment (4)
    if (nseg * DIV != ttbl::T_NROW) return fail(QM_ERR_INVALID, "Student t: %d segments", nseg);
    for (int j = 0; j < nseg; ++j) {
        const double* c = seg10 + 10 * j;
        for (int q = 0; q < DIV; ++q) {
            const int r = DIV * j + q;
            // the row start r/128 in the segment's variable s (about the centre,
            // or about 0 for j = 0): s = sigma + dl
            const LD dl = (LD)q / ttbl::T_ROWS_PER_UNIT - (j == 0 ? 0.0 : 1.0 / (2 * H_INV));
            LD cp[10];
            for (int m = 0; m < 10; ++m) {
                LD acc = 0, p = 1;
                for (int k = m; k < 10; ++k) {
                    acc += (LD)c[k] * binom[k][m] * p;
                    p *= dl;
                }
                cp[m] = acc;
            }
            // H in th = 64 sigma: b'_k = cp_{k+1} 64^-k, k = 0..6 (degree 7 in sigma)
            LD bh[7];
            for (int k = 0; k < 7; ++k) bh[k] = std::ldexp(cp[k + 1], -6 * k);
            if (!(bh[0] > 0)) return fail(QM_ERR_UNSUPPORTED, "Student t: row %d has a non-positive slope", r);
            for (int k = 1; k < 7; ++k) {
                if (bh[k] < 0) {
                    if (-bh[k] > 1e-18 * bh[0])
                        return fail(QM_ERR_UNSUPPORTED, "Student t: row %d coefficient %d negative", r, k);
                    bh[k] = 0;                                           // rounding residue
                }
            }
            LD hmax = 0;
            for (int k = 0; k < 7; ++k) hmax += std::ldexp(bh[k], -k);   // H at th = 1/2
            if (!(hmax < 2 * bh[0])) return fail(QM_ERR_UNSUPPORTED, "Student t: row %d varies too fast", r);
            int e2 = 0;
            std::frexp((double)bh[0], &e2);                              // b'_0 in [2^(e2-1), 2^e2)
            const int s0 = e2 - 1 - ttbl::T_HB;                           // H(0) 2^-s0 in [2^HB, 2^(HB+1))
            long long B[3];
            for (int k = 0; k < 3; ++k) B[k] = std::llround(std::ldexp(bh[k], -s0));
            const int e0 = 1022 + ttbl::T_HB + s0;
            // the outer accumulators stay below 2^62 (the high products' bound):
            // every partial Horner value at th = 1/2
            for (int k = 1; k <= 2; ++k) {
                LD part = 0;
                for (int i = k; i < 7; ++i) part += std::ldexp(bh[i], -(i - k));
                if (!(std::ldexp(part, -s0) < std::ldexp((LD)1, 62) - 64))
                    return fail(QM_ERR_UNSUPPORTED, "Student t: row %d partial sum %d out of range", r, k);
            }
            // inner chain: C_k = b'_{k+3} 2^-(s0 + cs) on 32-bit integers, cs the
            // smallest scale (at least 1) that keeps every Horner partial value
            // C_k + C_{k+1}/2 + ... (th < 1/2) below 2^32
            LD fk[4];
            for (int k = 0; k < 4; ++k) fk[k] = std::ldexp(bh[k + 3], -s0);
            auto partial_max = [](const LD* v) {
                LD m = 0;
                for (int k = 0; k < 4; ++k) {
                    LD acc = 0;
                    for (int i = 3; i >= k; --i) acc = acc * 0.5 + v[i];
                    m = std::max(m, acc);
                }
                return m;
            };
            int cs = 1;
            {
                const LD pm = partial_max(fk);
                if (pm > 0) cs = std::max(1, (int)std::ceil(std::log2((double)pm)) - 32);
            }
            long long C[4];
            for (;; ++cs) {
                LD cd[4];
                for (int k = 0; k < 4; ++k) {
                    C[k] = std::llround(std::ldexp(fk[k], -cs));
                    cd[k] = (LD)C[k];
                }
                if (partial_max(cd) < 4294967288.0 || cs > 32) break;
            }
            if (B[0] < (1ll << ttbl::T_HB) || B[2] >= (1ll << 52) || e0 <= 0 || e0 >= 2048 || cs > 32 ||
                C[3] >= (1ll << 27))
                return fail(QM_ERR_UNSUPPORTED, "Student t: row %d outside the fixed-point range", r);
            fxt::SegA& A = out->a[r];
            fxt::SegC& W = out->c[r];
            A.a0 = (double)cp[0];
            A.B0 = B[0];
            A.B1 = B[1];
            A.B2s = (long long)((unsigned long long)B[2] | ((unsigned long long)e0 << 52));
            W.c3 = (unsigned)C[0];
            W.c4 = (unsigned)C[1];
            W.c5 = (unsigned)C[2];
            W.c6s = (unsigned)C[3] | ((unsigned)(32 - cs) << 27);
            // the stored row against the original expansion (degree 9) at
            // points of the row: quantisation of a0, B_k and C_k, and the
            // truncation to degree 7
            for (int qq = 0; qq <= 4; ++qq) {
                const LD sig = (LD)qq / (4 * ttbl::T_ROWS_PER_UNIT) * (qq == 4 ? 1 - 1.0 / 4096 : 1);
                const LD th = 64 * sig, s = sig + dl;
                LD H = 0, ref = 0;
                for (int k = 6; k >= 0; --k)
                    H = H * th + (k < 3 ? std::ldexp((LD)B[k], s0) : std::ldexp((LD)C[k - 3], s0 + cs));
                for (int k = 9; k >= 0; --k) ref = ref * s + (LD)c[k];
                const LD got = (LD)A.a0 + sig * H;
                if (ref != 0 && std::fabs(got / ref - 1) > 1e-12)
                    return fail(QM_ERR_UNSUPPORTED, "Student t: row %d fixed-point form off by %g", r,
                                (double)std::fabs(got / ref - 1));
            }
        }
    }
    return QM_OK;
}

qm_status pack_fx_biased(const double* coef, double w, double h_in, ttbl::SegTX* out)
{
    using LD = long double;
    static const LD binom[10][10] = {
        {1}, {1, 1}, {1, 2, 1}, {1, 3, 3, 1}, {1, 4, 6, 4, 1}, {1, 5, 10, 10, 5, 1},
        {1, 6, 15, 20, 15, 6, 1}, {1, 7, 21, 35, 35, 21, 7, 1}, {1, 8, 28, 56, 70, 56, 28, 8, 1},
        {1, 9, 36, 84, 126, 126, 84, 36, 9, 1}};
    const LD h = (LD)h_in;
    LD cp[10];                                                   // about the start: s = sigma - h
    for (int m = 0; m < 10; ++m) {
        LD acc = 0, p = 1;
        for (int k = m; k < 10; ++k) {
            acc += (LD)coef[k] * binom[k][m] * p;
            p *= -h;
        }
        cp[m] = acc;
    }
    LD d[9];                                                     // P in tau = sigma / (2 w)
    for (int k = 0; k < 9; ++k) d[k] = cp[k + 1] * std::pow(2 * (LD)w, (LD)k);
    LD var = 0;                                                  // bound on |P - d_0| over tau < 1/2
    for (int k = 1; k < 9; ++k) var += std::fabs(d[k]) * std::ldexp((LD)1, -k);
    const LD pmin = d[0] - var, pmax = d[0] + var;
    if (!(pmin > 0) || !(pmax < 2 * pmin) || !std::isfinite((double)pmax))
        return fail(QM_ERR_UNSUPPORTED, "fixed-point row: P not within a factor 2 over the segment");
    int e2 = 0;
    std::frexp((double)pmin, &e2);                               // pmin in [2^(e2-1), 2^e2)
    const int s0 = e2 - 60;                                       // pmin 2^-s0 in [2^59, 2^60)
    // every partial Horner value of the outer steps below 2^60 in magnitude
    for (int k = 1; k <= 4; ++k) {
        LD part = 0;
        for (int i = k; i < 9; ++i) part += std::fabs(d[i]) * std::ldexp((LD)1, -(i - k));
        if (!(std::ldexp(part, -s0) < std::ldexp((LD)1, 60) - 64))
            return fail(QM_ERR_UNSUPPORTED, "fixed-point row: partial sum %d out of range", k);
    }
    long long D[5];
    for (int k = 0; k < 5; ++k) D[k] = std::llround(std::ldexp(d[k], -s0));
    const int e0 = 1081 + s0;
    if (e0 <= 0 || e0 >= 2048 || D[4] <= -(1ll << 51) || D[4] >= (1ll << 51))
        return fail(QM_ERR_UNSUPPORTED, "fixed-point row outside the exponent or D_4 range");
    // inner chain on 32-bit integers under the scale 2^c: |a_k| < 2^29 for
    // the partial values of C_5..C_7, |C_8| < 2^25
    LD f[4], pm = 0;
    for (int k = 0; k < 4; ++k) f[k] = std::ldexp(d[k + 5], -s0);
    for (int k = 0; k < 4; ++k) {
        LD part = 0;
        for (int i = k; i < 4; ++i) part += std::fabs(f[i]) * std::ldexp((LD)1, -(i - k));
        pm = std::max(pm, part);
    }
    int c = (pm > 0) ? std::max(1, (int)std::ceil(std::log2((double)pm)) - 28) : 1;
    long long C[4];
    for (;; ++c) {
        if (c > 32) return fail(QM_ERR_UNSUPPORTED, "fixed-point row: inner chain out of range");
        for (int k = 0; k < 4; ++k) C[k] = std::llround(std::ldexp(f[k], -c));
        LD pmc = 0;
        for (int k = 0; k < 4; ++k) {
            LD part = 0;
            for (int i = k; i < 4; ++i) part += std::fabs((LD)C[i]) * std::ldexp((LD)1, -(i - k));
            pmc = std::max(pmc, part);
        }
        if (pmc < (LD)((1ll << 29) - 16) && C[3] > -(1ll << 25) && C[3] < (1ll << 25)) break;
    }
    ttbl::SegTX& r = *out;
    r.a0 = (double)cp[0];
    r.D0 = (unsigned long long)D[0];
    r.D1 = (unsigned long long)(D[1] + (1ll << 60));
    r.D2 = (unsigned long long)(D[2] + (1ll << 60));
    r.D3 = (unsigned long long)(D[3] + (1ll << 60));
    r.D4e = (unsigned long long)(D[4] + (1ll << 51)) | ((unsigned long long)e0 << 52);
    for (int k = 0; k < 3; ++k) r.c[k] = (unsigned)(C[k] + (1ll << 29));
    r.c[3] = (unsigned)(C[3] + (1ll << 25)) | ((unsigned)(32 - c) << 27);
    // the packed form against the original expansion at points of the segment
    for (int q = 0; q <= 4; ++q) {
        const LD sig = (LD)w * q / 4 * (q == 4 ? (1 - 1.0L / 4096) : 1);
        const LD tau = sig / (2 * (LD)w), sc = sig - h;
        LD P = 0, ref = 0;
        for (int k = 8; k >= 0; --k)
            P = P * tau + (k < 5 ? std::ldexp((LD)D[k], s0) : std::ldexp((LD)C[k - 5], s0 + c));
        for (int k = 9; k >= 0; --k) ref = ref * sc + (LD)coef[k];
        const LD got = (LD)r.a0 + sig * P;
        if (ref != 0 && std::fabs(got / ref - 1) > 1e-13L)
            return fail(QM_ERR_UNSUPPORTED, "fixed-point row off by %g", (double)std::fabs(got / ref - 1));
    }
    return QM_OK;
}

namespace {

struct Entry {
    int device;
    double nu;
    ttbl::TRows* seg;    // device, the fixed-point rows
    double* tail;        // device, 3 + NT doubles
};

std::mutex g_mu;
std::vector<Entry> g_cache;
constexpr size_t kMaxEntries = 256;

}  // namespace

// Device tables for nu on the current device, built and uploaded at first use.
qm_status t_table_device(double nu, const void** seg_dev, const double** tail_dev)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return fail(QM_ERR_CUDA, "Student t: no current device");
    std::lock_guard<std::mutex> lk(g_mu);
    for (const Entry& e : g_cache)
        if (e.device == dev && e.nu == nu) {
            *seg_dev = e.seg;
            *tail_dev = e.tail;
            return QM_OK;
        }
    if (g_cache.size() >= kMaxEntries)
        return fail(QM_ERR_NOMEM, "Student t: more than %zu distinct nu in use", kMaxEntries);
    std::vector<double> seg(10 * NSEG), tail(3 + NT);
    const qm_status st = t_table_build(nu, seg.data(), tail.data());
    if (st != QM_OK) return st;
    std::vector<ttbl::TRows> packed(1);
    const qm_status pst = t_pack_rows(seg.data(), NSEG, packed.data());
    if (pst != QM_OK) return pst;
    Entry e{dev, nu, nullptr, nullptr};
    if (cudaMalloc(&e.seg, sizeof(ttbl::TRows)) != cudaSuccess ||
        cudaMalloc(&e.tail, sizeof(double) * tail.size()) != cudaSuccess) {
        if (e.seg) cudaFree(e.seg);
        return fail(QM_ERR_NOMEM, "Student t: table allocation failed");
    }
    if (cudaMemcpy(e.seg, packed.data(), sizeof(ttbl::TRows), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(e.tail, tail.data(), sizeof(double) * tail.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(e.seg);
        cudaFree(e.tail);
        return fail(QM_ERR_CUDA, "Student t: table upload failed");
    }
    g_cache.push_back(e);
    *seg_dev = e.seg;
    *tail_dev = e.tail;
    return QM_OK;
}

namespace {

// The offline tables of the tabulated nu, as device pointers: the segments of
// this module's SEG_T read back once per device and converted to the
// fixed-point rows (NNU x NSEG), the tail (nu, log kappa, TAIL_DEG, R_k) in a
// small buffer; both built once per device and kept until exit.
struct StaticT {
    int device;
    ttbl::TRows* seg;      // NNU row tables
    double* tail;          // NNU x (3 + TAIL_DEG + 1)
};
std::vector<StaticT> g_static;
constexpr int kStaticTail = 3 + ttbl::TAIL_DEG + 1;

qm_status static_tables(int dev, const StaticT** out)
{
    for (const StaticT& e : g_static)
        if (e.device == dev) {
            *out = &e;
            return QM_OK;
        }
    StaticT e{dev, nullptr, nullptr};
    std::vector<ttbl::SegT> offline(ttbl::NNU * NSEG);
    if (cudaMemcpyFromSymbol(offline.data(), ttbl::SEG_T, sizeof(ttbl::SegT) * offline.size()) != cudaSuccess)
        return fail(QM_ERR_CUDA, "Student t: table read failed");
    std::vector<double> seg10(10 * NSEG);
    std::vector<ttbl::TRows> packed(ttbl::NNU);
    for (int k = 0; k < ttbl::NNU; ++k) {
        for (int j = 0; j < NSEG; ++j) {
            const ttbl::SegT& g = offline[k * NSEG + j];
            for (int c = 0; c < 5; ++c) seg10[10 * j + c] = g.a[c];
            for (int c = 0; c < 5; ++c) seg10[10 * j + 5 + c] = g.b[c];
        }
        const qm_status pst = t_pack_rows(seg10.data(), NSEG, packed.data() + k);
        if (pst != QM_OK) return pst;
    }
    double kappa[ttbl::NNU], rt[ttbl::NNU][ttbl::TAIL_DEG + 1];
    if (cudaMemcpyFromSymbol(kappa, ttbl::T_KAPPA, sizeof(kappa)) != cudaSuccess ||
        cudaMemcpyFromSymbol(rt, ttbl::T_TAIL, sizeof(rt)) != cudaSuccess)
        return fail(QM_ERR_CUDA, "Student t: table read failed");
    std::vector<double> tail(ttbl::NNU * kStaticTail);
    for (int k = 0; k < ttbl::NNU; ++k) {
        double* t = &tail[k * kStaticTail];
        t[0] = ttbl::T_NU[k];
        t[1] = std::log(kappa[k]);
        t[2] = ttbl::TAIL_DEG;
        for (int c = 0; c <= ttbl::TAIL_DEG; ++c) t[3 + c] = rt[k][c];
    }
    if (cudaMalloc(&e.tail, sizeof(double) * tail.size()) != cudaSuccess)
        return fail(QM_ERR_NOMEM, "Student t: table allocation failed");
    if (cudaMalloc(&e.seg, sizeof(ttbl::TRows) * packed.size()) != cudaSuccess) {
        cudaFree(e.tail);
        return fail(QM_ERR_NOMEM, "Student t: table allocation failed");
    }
    if (cudaMemcpy(e.tail, tail.data(), sizeof(double) * tail.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(e.seg, packed.data(), sizeof(ttbl::TRows) * packed.size(), cudaMemcpyHostToDevice) !=
            cudaSuccess) {
        cudaFree(e.tail);
        cudaFree(e.seg);
        return fail(QM_ERR_CUDA, "Student t: table upload failed");
    }
    g_static.push_back(e);
    *out = &g_static.back();
    return QM_OK;
}

}  // namespace

qm_status t_select(double nu, int* k, const void** seg_dev, const double** tail_dev)
{
    *seg_dev = nullptr;
    *tail_dev = nullptr;
    for (int i = 0; i < ttbl::NNU; ++i)
        if (nu == ttbl::T_NU[i]) {
            *k = i;
            int dev = 0;
            if (cudaGetDevice(&dev) != cudaSuccess) return fail(QM_ERR_CUDA, "Student t: no current device");
            std::lock_guard<std::mutex> lk(g_mu);
            const StaticT* st = nullptr;
            const qm_status s = static_tables(dev, &st);
            if (s != QM_OK) return s;
            *seg_dev = st->seg + i;
            *tail_dev = st->tail + i * kStaticTail;
            return QM_OK;
        }
    *k = -1;
    if (!(nu > 0.0)) return fail(QM_ERR_INVALID, "Student t: nu must be > 0 (got %g)", nu);
    if (!(nu >= QM_T_NU_MIN && nu <= QM_T_NU_MAX))
        return fail(QM_ERR_UNSUPPORTED, "Student t: nu = %g outside [%g, %g] and not tabulated", nu,
                    QM_T_NU_MIN, QM_T_NU_MAX);
    return t_table_device(nu, seg_dev, tail_dev);
}

}  // namespace qm

extern "C" qm_status qm_t_table_build(double nu, double* seg_coef, double* tail)
{
    if (!seg_coef || !tail) return qm::fail(QM_ERR_INVALID, "qm_t_table_build: null pointer");
    return qm::t_table_build(nu, seg_coef, tail);
}

extern "C" qm_status qm_t_rows_build(double nu, void* rows)
{
    if (!rows) return qm::fail(QM_ERR_INVALID, "qm_t_rows_build: null pointer");
    std::vector<double> seg(10 * QM_T_NSEG), tail(3 + QM_T_TAIL_TERMS);
    const qm_status st = qm::t_table_build(nu, seg.data(), tail.data());
    if (st != QM_OK) return st;
    return qm::t_pack_rows(seg.data(), QM_T_NSEG, static_cast<qm::ttbl::TRows*>(rows));
}
