// qm_fx.cuh -- layout of the fixed-point FP64 segment table and its
// evaluation (the FIXED normal quantile; table data in qm_fx_tables.h,
// generated by fit/gen_fx_tables.py, compiled into qm_fixed.cu only; other
// translation units get its device address from fx_table_device()).
//
// Phi^{-1}(u) through the paper's change of variable v = -log(2d),
// d = min(u, 1-u) (Sec. 6, Sec. 7.2), without forming v: x = 2d = M 2^(E-52)
// with a 53-bit integer significand M; (E, top K bits of M) select a segment
// whose local expansion G of Q(v) = Phi^{-1}(1 - e^{-v}/2) comes from the
// recycling ODE Q'' + Q' = Q Q'^2 (Sec. 2.3, Sec. 6).  With the offset
// t_u = T 2^-52 > 0 back from the segment's end (T an exact integer; the end
// of the top segment is x = 1, where z = 0) and tau = t_u 2^K in (0, 1]:
//
//     |z| = a0 + t_u H,   H = beta_0 + tau (beta_1 + tau (beta_2 + tau F)) > 0,
//     F   = beta_3 + tau (beta_4 + tau (beta_5 + tau beta_6))   (single precision)
//
// The Horner steps for beta_0..beta_2 run on signed 64-bit accumulators times
// tau as an unsigned Q0.64 integer (unsigned mulhi plus a sign correction),
// the normalisation of x is integer arithmetic, and t_u and H become doubles
// by bit assembly, so the only FP64 instruction is the final FMA.
#pragma once
#include <stdint.h>

namespace qm {
namespace fxt {

constexpr int K_MAIN = 6;
constexpr int E_MAIN = 64;
constexpr int K_DEEP = 5;
constexpr int E_LAST = 1072;
constexpr int N_MAIN = 4096;
constexpr int N_ALL = 36384;

struct alignas(64) SegFx {
    double a0;
    long long B0, B1, B2;
    float f3, f4, f5, f6;
    int s0;
    float csc;
    int sh;
    int pad;
};

}  // namespace fxt

// 32 bytes from the read-only path in one 256-bit load
__device__ __forceinline__ void ld256(const void* p, unsigned long long& a, unsigned long long& b,
                                      unsigned long long& c, unsigned long long& d)
{
    asm("ld.global.nc.v4.u64 {%0, %1, %2, %3}, [%4];"
        : "=l"(a), "=l"(b), "=l"(c), "=l"(d) : "l"(p));
}

// floor(a b / 2^64) for signed a and unsigned b
__device__ __forceinline__ long long mulhi_su(long long a, unsigned long long b)
{
    const unsigned long long h = __umul64hi((unsigned long long)a, b);
    return (long long)(h - (a < 0 ? b : 0ull));
}

// |Phi^{-1}| bits for x = 2d = S 2^(base - 52), 0 < S < 2^53 (any position of
// the leading bit), from the table T (x = 1, i.e. d = 1/2, gives +0).
__device__ __forceinline__ unsigned long long probit_mag_fx_sx(const fxt::SegFx* T, unsigned long long S,
                                                             int base)
{
    const int lz = __clzll(S | 1ull) - 11;
    const unsigned long long Mx = S << lz;                      // 2^52 <= Mx < 2^53
    const int e = -1 - (base - lz);                             // binade: x in [2^-e-1, 2^-e)
    const int ec = min(max(e, 0), fxt::E_LAST);
    const bool mainb = ec < fxt::E_MAIN;
    const int K = mainb ? fxt::K_MAIN : fxt::K_DEEP;
    const int sK = 52 - K;
    const unsigned j = (unsigned)(Mx >> sK) & ((1u << K) - 1u);
    const int idx = mainb ? (ec << fxt::K_MAIN) + (int)j
                          : fxt::N_MAIN + ((ec - fxt::E_MAIN) << fxt::K_DEEP) + (int)j;
    // offset back from the segment end: Tu in [1, 2^sK]
    const unsigned long long Tu = (1ull << sK) - (Mx & ((1ull << sK) - 1ull));
    const unsigned long long Tau = (Tu << (12 + K)) - (Tu >> sK);   // tau 2^64 (tau = 1 -> 1 - 2^-64)

    const fxt::SegFx* p = T + idx;
    unsigned long long a0b, B0, B1, B2, f34, f56, s0c, shp;
    ld256(p, a0b, B0, B1, B2);                                     // a0, B0, B1, B2
    ld256(reinterpret_cast<const char*>(p) + 32, f34, f56, s0c, shp);   // beta_3..6, s0, 2^c, sh

    // single-precision tail from the top bits of the offset
    const float tf = __uint_as_float(0x4B000000u | (unsigned)(Tu >> 25)) - 8388608.0f;
    const float tau_f = tf * __uint_as_float((unsigned)(127 + K - 27) << 23);
    float F = __fmaf_rn(__uint_as_float((unsigned)(f56 >> 32)), tau_f, __uint_as_float((unsigned)f56));
    F = __fmaf_rn(F, tau_f, __uint_as_float((unsigned)(f34 >> 32)));
    F = __fmaf_rn(F, tau_f, __uint_as_float((unsigned)f34));
    const int i3 = __float2int_rn(F * __uint_as_float((unsigned)(s0c >> 32)));
    long long acc = (long long)((unsigned long long)(long long)i3 << (unsigned)shp);
    acc = (long long)B2 + mulhi_su(acc, Tau);
    acc = (long long)B1 + mulhi_su(acc, Tau);
    acc = (long long)B0 + mulhi_su(acc, Tau);                     // H 2^-s0, in (0, 2^62)

    // H as a double: normalise, round to 53 bits, insert the exponent
    const unsigned long long ha = (unsigned long long)acc;
    const int lh = __clzll(ha);
    const unsigned long long hm = ((ha << lh) + 0x400ull) >> 11;
    const unsigned long long hbits = hm + ((unsigned long long)(1022 + 63 - lh + (int)(unsigned)s0c) << 52);
    // t_u as a double (exact: 1 <= Tu <= 2^47)
    const int lt = __clzll(Tu);
    const unsigned long long tbits = (Tu << (lt - 11)) + ((unsigned long long)(1033 - lt) << 52);
    const double g = __fma_rn(__longlong_as_double((long long)tbits),
                              __longlong_as_double((long long)hbits), __longlong_as_double((long long)a0b));
    return (e < 0) ? 0ull : (unsigned long long)__double_as_longlong(g);
}


// |Phi^{-1}(u)| bits for 0 < u < 1 (other inputs give an unused value; the
// table index is in range for every bit pattern).  x = 2d = S 2^(base - 52):
// u >= 1/2 -> S = 2^52 - frac (1 - u exact), u < 1/2 -> S = significand of u
// (no implicit bit when subnormal).
__device__ __forceinline__ unsigned long long probit_mag_fx(const fxt::SegFx* T, unsigned long long ub)
{
    const bool upper = ub >= 0x3FE0000000000000ull;
    const unsigned long long frac = ub & 0x000FFFFFFFFFFFFFull;
    const int eb = (int)(ub >> 52) & 0x7ff;
    const unsigned long long S = upper ? (1ull << 52) - frac : (eb ? (frac | (1ull << 52)) : frac);
    const int base = upper ? 0 : max(eb, 1) - 1022;
    return probit_mag_fx_sx(T, S, base);
}

// |Phi^{-1}((k + 1/2) 2^-53)| for a 53-bit integer k on its exact reflected
// grid point d = (min(k, 2^53-1-k) + 1/2) 2^-53: x = 2d = (2j+1) 2^-53;
// upper = (k >= 2^52), the sign of z.
__device__ __forceinline__ double probit_grid53_fx(const fxt::SegFx* T, unsigned long long k, bool& upper)
{
    upper = k >= (1ull << 52);
    const unsigned long long j = upper ? ((1ull << 53) - 1 - k) : k;
    return __longlong_as_double((long long)probit_mag_fx_sx(T, 2 * j + 1, -1));
}

// Phi^{-1}(u) with the IEEE edge values: u = 1/2 -> +0, u = 0 -> -inf,
// u = 1 -> +inf, NaN or u outside [0, 1] -> NaN.
__device__ __forceinline__ double probit_fx(const fxt::SegFx* T, double u)
{
    const unsigned long long ub = (unsigned long long)__double_as_longlong(u);
    const unsigned hi = (unsigned)(ub >> 32);
    const unsigned long long mb = probit_mag_fx(T, ub);
    const bool valid = hi < 0x3FF00000u && ub != 0ull;                    // 0 < u < 1
    const unsigned sgn = hi < 0x3FE00000u ? 0x80000000u : 0u;              // u < 1/2
    const unsigned sp = ((ub << 1) == 0ull) ? 0xfff00000u                  // +-0 -> -inf
                      : (ub == 0x3FF0000000000000ull ? 0x7ff00000u         // 1 -> +inf
                                                     : 0x7ff80000u);       // NaN
    const unsigned rhi = valid ? ((unsigned)(mb >> 32) | sgn) : sp;
    const unsigned rlo = valid ? (unsigned)mb : 0u;
    return __hiloint2double((int)rhi, (int)rlo);
}


}  // namespace qm
