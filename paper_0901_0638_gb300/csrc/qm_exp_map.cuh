// qm_exp_map.cuh -- table-driven exponential -> normal recycling map
// z = Phi^{-1}(1 - e^{-x}) (Sec. 2.3, Sec. 6) on given samples x.
// Regions (tables and their construction: fit/gen_exp_tables.py):
//   x >= ln 2              z = Q(v), v = x - ln 2         (V table, s = v - v_c)
//   ln2 - 1/64 < x < ln 2  z = -H(y), y = ln 2 - x        (one series at y = 0)
//   2^-26 <= x             z = -F(r), x = 2^E m, r = m c - 1 (X table)
//   x < 2^-26              z = -|Phi^{-1}|(x - x^2/2)     (normal table on u)
// Include in the translation units that use it (tables are per unit).
#pragma once

#include "qm_device.cuh"
#include "qm_exp_tables.h"

namespace qm {

// (2q + 1) 2^-p as a double, built from its bits (q >= 0).
__device__ __forceinline__ double odd_scaled(uint32_t q, int p)
{
    const uint32_t odd = 2u * q + 1u;
    const int lz = 31 - __clz(odd);
    const uint64_t bits = ((uint64_t)(lz - p + 1023) << 52) |
                          (((uint64_t)odd << (52 - lz)) & 0x000fffffffffffffull);
    return __longlong_as_double((long long)bits);
}

// a0..a4 in double, a5..a9 in single precision (their terms are below 1e-6
// of the result), Horner in s.
__device__ __forceinline__ double segT_eval(const ttbl::SegT& g, double s)
{
    const float sf = dtof_trunc(s);
    float tf = __fmaf_rn(g.b[4], sf, g.b[3]);
    tf = __fmaf_rn(tf, sf, g.b[2]);
    tf = __fmaf_rn(tf, sf, g.b[1]);
    tf = __fmaf_rn(tf, sf, g.b[0]);
    double acc = __fma_rn(ftod_exact(tf), s, g.a[4]);
    acc = __fma_rn(acc, s, g.a[3]);
    acc = __fma_rn(acc, s, g.a[2]);
    acc = __fma_rn(acc, s, g.a[1]);
    return __fma_rn(acc, s, g.a[0]);
}

static __device__ __noinline__ double exp_to_normal_edge(double x)
{
    if (x == 0.0) return __longlong_as_double(0xfff0000000000000ll);      // -inf (also -0)
    if (x == __longlong_as_double(0x7ff0000000000000ll)) return x;          // +inf
    return __longlong_as_double(0x7ff8000000000000ll);                     // x < 0, NaN
}

__device__ __forceinline__ double exp_to_normal_tbl(double x)
{
    const uint64_t xb = (uint64_t)__double_as_longlong(x);
    if (xb == 0 || xb >= 0x7ff0000000000000ull) return exp_to_normal_edge(x);
    const double kLn2Hi = 0.69314718055994528623, kLn2Lo = 2.3190468138462996154e-17;
    const double y = __dadd_rn(__dadd_rn(kLn2Hi, -x), kLn2Lo);
    if (y <= 0.0) {
        const double v = -y;
        const uint64_t vb = (uint64_t)__double_as_longlong(v);
        if (vb >= 0x4050000000000000ull) return probit_mag_exp_deep(v);   // v >= 64
        const int E = (int)(vb >> 52) - 1023;
        const uint64_t M = (vb & 0x000fffffffffffffull) | (1ull << 52);
        uint32_t j;
        double vc;
        if (E < 0) {                                                       // v < 1: width 1/32
            j = (E + 5 < 0) ? 0u : (uint32_t)(M >> (52 - (E + 5)));
            vc = (j == 0) ? 0.0 : odd_scaled(j, 6);
        } else {                                                           // width 1/8
            const uint32_t q = (uint32_t)(M >> (52 - (E + 3)));            // floor(8 v) >= 8
            j = q + (etbl::V_FINE * etbl::V_SPLIT - etbl::V_COARSE * etbl::V_SPLIT);
            vc = odd_scaled(q, 4);
        }
        if (vb == 0) return 0.0;
        return segT_eval(etbl::SEG_V[j], __dadd_rn(v, -vc));
    }
    if (y < 1.0 / etbl::Y_MAX_INV) {
        double h = etbl::Y_SERIES[etbl::DEG_Y];
#pragma unroll
        for (int k = etbl::DEG_Y - 1; k >= 0; --k) h = __fma_rn(h, y, etbl::Y_SERIES[k]);
        return -h;
    }
    if (xb >= 0x3E50000000000000ull) {                                     // x >= 2^-26
        const int E = (int)(xb >> 52) - 1023;                              // -26 .. -1
        const int j = (int)((xb >> (52 - etbl::X_K)) & ((1u << etbl::X_K) - 1));
        const double m = __longlong_as_double((long long)((xb & 0x000fffffffffffffull) | 0x3ff0000000000000ull));
        return -f64_seg_eval(&etbl::SEG_X[(-1 - E) * (1 << etbl::X_K) + j], m);
    }
    // x < 2^-26: u = 1 - e^{-x} = x - x^2/2 to double precision
    const double u = __fma_rn(-0.5 * x, x, x);
    const double mag = f64_tbl_covers(u) ? probit_mag_f64_tbl(u) : probit_mag_exp_deep(-log(2.0 * u));
    return -mag;
}

}  // namespace qm
