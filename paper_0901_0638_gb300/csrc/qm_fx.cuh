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
// t_u = T 2^-52 > 0 back from the segment's end (T in [1, 2^(52-K)] an exact
// integer; the end of the top segment is x = 1, where z = 0), H is stored as
// a polynomial in tau' = (T - 1) 2^(K-52) in [0, 1) (the expansion in
// t_u 2^K moved by one unit of T, so that tau' 2^64 fits 64 bits and T - 1
// is the complement of the significand's low bits):
//
//     |z| = a0 + t_u H,   H = beta_0 + tau' (beta_1 + tau' (beta_2 + tau' F)) > 0,
//     F   = beta_3 + tau' (beta_4 + tau' (beta_5 + tau' beta_6))   (single precision)
//
// The Horner steps for beta_0 and beta_1 run on signed 64-bit accumulators
// times tau' as an unsigned Q0.64 integer (unsigned mulhi plus a sign
// correction); beta_3..beta_6 are stored pre-scaled to the accumulator's
// units, and the single-precision chain F enters the beta_2 step as
// B2 + rn(F tau'), F tau' formed in single precision from an exact two-float
// split of tau'.  The
// normalisation of x is integer arithmetic, H becomes a double by bit
// assembly and t_u exactly (two instruction mixes, below), and the final FMA
// is the one FP64 operation of the method.  A segment is 48 bytes in two
// arrays (one 256-bit and one 128-bit gather per element; the denser arrays
// also put more segments in a cache line).
#pragma once
#include <stdint.h>

namespace qm {
namespace fxt {

constexpr int K = 6;           // 64 segments in every binade
constexpr int E_LAST = 1072;   // binades e = -1 - E = 0 .. 1072 (x down to 2^-1073)
constexpr int N_ALL = (E_LAST + 1) << K;

// a0, B0 = beta_0 2^-s0, B1 = beta_1 2^-s0, and B2 = beta_2 2^-s0 in the low
// 52 bits (sign extended) with s0 in the top 12
struct alignas(32) SegA {
    double a0;
    long long B0, B1, B2s;
};

// f_k = beta_k 2^-s0, k = 3..6, rounded to single precision
struct alignas(16) SegF {
    float f3, f4, f5, f6;
};

struct FxTable {
    SegA a[N_ALL];
    SegF f[N_ALL];
};

}  // namespace fxt

// 32 bytes from the read-only path in one 256-bit load
__device__ __forceinline__ void ld256(const void* p, unsigned long long& a, unsigned long long& b,
                                      unsigned long long& c, unsigned long long& d)
{
    asm("ld.global.nc.v4.u64 {%0, %1, %2, %3}, [%4];"
        : "=l"(a), "=l"(b), "=l"(c), "=l"(d) : "l"(p));
}

// 16 bytes from the read-only path in one 128-bit load
__device__ __forceinline__ float4 ld128f(const void* p)
{
    float4 v;
    asm("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
    return v;
}

// float -> int64 rounded to nearest even, by integer operations: the same
// value as __float2ll_rn for |F| < 2^62 (the hardware conversion to 64 bits
// issues on the FP64 pipe).
__device__ __forceinline__ long long f32_to_i64_rn_alu(float F)
{
    const unsigned b = __float_as_uint(F);
    const int ex = (int)((b >> 23) & 0xFFu);
    const unsigned m = (b & 0x7FFFFFu) | 0x800000u;          // (zero: rounds to 0 below)
    unsigned long long mag;
    if (ex >= 150) {
        mag = (unsigned long long)m << (ex - 150);             // already an integer
    } else {
        const int r = min(150 - ex, 25);                       // 1 .. 25
        const unsigned q = m >> r;
        const unsigned rem = m & ((1u << r) - 1u);
        const unsigned half = 1u << (r - 1);
        mag = q + (unsigned)((rem > half) | ((rem == half) & ((q & 1u) != 0u)));
    }
    return (b >> 31) ? -(long long)mag : (long long)mag;
}

// Instruction mixes with bit-identical results, chosen per kernel by what
// bounds it (two steps can run on the FP64 pipe or as integer operations):
//   FX_CVT_HW  -- the float -> int64 conversion by the hardware instruction
//                 (one FP64-pipe slot) instead of f32_to_i64_rn_alu;
//   FX_TU_FADD -- t_u as (1 + t_u) - 1, one exact FP64 add, instead of
//                 normalising Tu with integer operations.
//   FX_INT_LEAN  = both (the streaming kernel, bound by the integer pipe and
//                  the L1: three FP64-pipe instructions per element);
//   FX_FP64_LEAN = neither (kernels bound by the FP64 pipe: the final FMA is
//                  the only FP64 instruction).
enum { FX_CVT_HW = 1, FX_TU_FADD = 2, FX_INT_LEAN = 3, FX_FP64_LEAN = 0 };

// floor(a b / 2^64) for signed a and unsigned b
__device__ __forceinline__ long long mulhi_su(long long a, unsigned long long b)
{
    const unsigned long long h = __umul64hi((unsigned long long)a, b);
    return (long long)(h - (a < 0 ? b : 0ull));
}

// |Phi^{-1}| bits for x = 2d = S 2^(base - 52), 0 < S < 2^53 (any position of
// the leading bit), from the table T (x = 1, i.e. d = 1/2, gives +0).
template <int MIX = FX_INT_LEAN>
__device__ __forceinline__ unsigned long long probit_mag_fx_sx(const fxt::FxTable* T, unsigned long long S,
                                                             int base)
{
    constexpr int K = fxt::K, sK = 52 - K;
    const int lz = __clzll(S | 1ull) - 11;
    const unsigned long long Mx = S << lz;                      // 2^52 <= Mx < 2^53
    const int e = -1 - (base - lz);                             // binade: x in [2^-e-1, 2^-e)
    const int ec = min(max(e, 0), fxt::E_LAST);
    const unsigned j = (unsigned)(Mx >> sK) & ((1u << K) - 1u);
    const int idx = (ec << K) + (int)j;
    // offset back from the segment end, Tu = Tp + 1 in [1, 2^sK]: Tp is the
    // complement of the significand's low sK bits.  H is stored in
    // tau' = Tp 2^-sK in [0, 1) (re-expanded by one unit of the offset), so
    // tau' 2^64 is a plain shift that never overflows.
    const unsigned long long Tp = ~Mx & ((1ull << sK) - 1ull);
    const unsigned long long Tau = Tp << (12 + K);

    unsigned long long a0b, B0, B1, B2s;
    ld256(&T->a[idx], a0b, B0, B1, B2s);                           // a0, B0, B1, B2 | s0
    const float4 f = ld128f(&T->f[idx]);                            // f3..f6
    const long long B2 = (long long)(B2s << 12) >> 12;
    const int s0 = (int)((long long)B2s >> 52);

    // single-precision tail from the top bits of the offset
    const float tf = __uint_as_float(0x4B000000u | (unsigned)(Tp >> 25)) - 8388608.0f;
    const float tau_f = tf * __uint_as_float((unsigned)(127 + K - 27) << 23);
    float F = __fmaf_rn(f.w, tau_f, f.z);
    F = __fmaf_rn(F, tau_f, f.y);
    F = __fmaf_rn(F, tau_f, f.x);
    // innermost step in single precision: tau' = Tp 2^-46 = th 2^-23 + tl 2^-46
    // exactly (both halves are integers below 2^23),
    // F tau' = fl(fl(F 2^-23 th) + F 2^-46 tl); acc = B2 + rn(F tau')
    const float th = __uint_as_float(0x4B000000u | (unsigned)(Tp >> 23)) - 8388608.0f;
    const float tl = __uint_as_float(0x4B000000u | ((unsigned)Tp & 0x7FFFFFu)) - 8388608.0f;
    const float f23 = F * 1.1920928955078125e-07f;                 // 2^-23, exact
    const float G = __fmaf_rn(f23 * 1.1920928955078125e-07f, tl, __fmul_rn(f23, th));
    long long acc = B2 + ((MIX & FX_CVT_HW) ? __float2ll_rn(G) : f32_to_i64_rn_alu(G));
    acc = (long long)B1 + mulhi_su(acc, Tau);
    acc = (long long)B0 + mulhi_su(acc, Tau);                     // H 2^-s0, in (0, 2^62)

    // H as a double: normalise, round to 53 bits, insert the exponent
    const unsigned long long ha = (unsigned long long)acc;
    const int lh = __clzll(ha);
    const unsigned long long hm = ((ha << lh) + 0x400ull) >> 11;
    const unsigned long long hbits = hm + ((unsigned long long)(1022 + 63 - lh + s0) << 52);
    // t_u as a double (exact, 1 <= Tu <= 2^sK): 1 + t_u has the bits
    // 0x3FF0... + Tu and taking 1 away again is exact (Sterbenz); or by
    // normalising Tu and inserting the exponent
    double tu;
    if (MIX & FX_TU_FADD) {
        tu = __dadd_rn(__longlong_as_double((long long)(0x3FF0000000000001ull + Tp)), -1.0);
    } else {
        const unsigned long long Tu = Tp + 1ull;
        const int lt = __clzll(Tu);
        tu = __longlong_as_double((long long)((Tu << (lt - 11)) + ((unsigned long long)(1033 - lt) << 52)));
    }
    const double g = __fma_rn(tu, __longlong_as_double((long long)hbits), __longlong_as_double((long long)a0b));
    return (e < 0) ? 0ull : (unsigned long long)__double_as_longlong(g);
}


// |Phi^{-1}(u)| bits for 0 < u < 1 (other inputs give an unused value; the
// table index is in range for every bit pattern).  x = 2d = S 2^(base - 52):
// u >= 1/2 -> S = 2^52 - frac (1 - u exact), u < 1/2 -> S = significand of u
// (no implicit bit when subnormal).
template <int MIX = FX_INT_LEAN>
__device__ __forceinline__ unsigned long long probit_mag_fx(const fxt::FxTable* T, unsigned long long ub)
{
    const bool upper = ub >= 0x3FE0000000000000ull;
    const unsigned long long frac = ub & 0x000FFFFFFFFFFFFFull;
    const int eb = (int)(ub >> 52) & 0x7ff;
    const unsigned long long S = upper ? (1ull << 52) - frac : (eb ? (frac | (1ull << 52)) : frac);
    const int base = upper ? 0 : max(eb, 1) - 1022;
    return probit_mag_fx_sx<MIX>(T, S, base);
}

// |Phi^{-1}((k + 1/2) 2^-53)| for a 53-bit integer k on its exact reflected
// grid point d = (min(k, 2^53-1-k) + 1/2) 2^-53: x = 2d = (2j+1) 2^-53;
// upper = (k >= 2^52), the sign of z.
template <int MIX = FX_INT_LEAN>
__device__ __forceinline__ double probit_grid53_fx(const fxt::FxTable* T, unsigned long long k, bool& upper)
{
    upper = k >= (1ull << 52);
    const unsigned long long j = upper ? ((1ull << 53) - 1 - k) : k;
    return __longlong_as_double((long long)probit_mag_fx_sx<MIX>(T, 2 * j + 1, -1));
}

// Phi^{-1}(u) with the IEEE edge values: u = 1/2 -> +0, u = 0 -> -inf,
// u = 1 -> +inf, NaN or u outside [0, 1] -> NaN.
template <int MIX = FX_INT_LEAN>
__device__ __forceinline__ double probit_fx(const fxt::FxTable* T, double u)
{
    const unsigned long long ub = (unsigned long long)__double_as_longlong(u);
    const unsigned hi = (unsigned)(ub >> 32);
    const unsigned long long mb = probit_mag_fx<MIX>(T, ub);
    const bool valid = hi < 0x3FF00000u && ub != 0ull;                    // 0 < u < 1
    const unsigned sgn = hi < 0x3FE00000u ? 0x80000000u : 0u;              // u < 1/2
    const unsigned sp = (((hi & 0x7fffffffu) | (unsigned)ub) == 0u) ? 0xfff00000u   // +-0 -> -inf
                      : (ub == 0x3FF0000000000000ull ? 0x7ff00000u         // 1 -> +inf
                                                     : 0x7ff80000u);       // NaN
    const unsigned rhi = valid ? ((unsigned)(mb >> 32) | sgn) : sp;
    const unsigned rlo = valid ? (unsigned)mb : 0u;
    return __hiloint2double((int)rhi, (int)rlo);
}


}  // namespace qm
