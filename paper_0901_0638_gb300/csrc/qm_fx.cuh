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
// t_u 2^K moved by one unit of T, so that T - 1 is the complement of the
// significand's low bits).  Every beta_k is positive (the tail quantile, as a
// function of the offset back from the segment end, has all derivatives
// positive), so the polynomial is evaluated in the half offset
// th = tau'/2 in [0, 1/2) on unsigned integers:
//
//     |z| = a0 + t_u H,   H = b0 + th (b1 + th (b2 + th F)) > 0,   b_k = beta_k 2^k,
//     F   = b3 + th (b4 + th (b5 + th b6))   (single precision)
//
// The Horner steps for b0 and b1 run on unsigned 64-bit accumulators (below
// 2^62) times th as a Q0.64 integer (below 2^63): the 128-bit product's high
// half is exact from four 32 x 32 -> 64-bit multiply-adds, none of which
// carries out.  b3..b6 are stored pre-scaled to the accumulator's units, and
// the single-precision chain F enters the b2 step as B2 + rn(F th), F th
// formed in single precision from an exact two-float split of th and turned
// into an integer exactly (rounding to nearest even) as two 24-bit halves by
// single-precision conversions.  The normalisation of x is integer
// arithmetic, H becomes a double by bit assembly and t_u exactly (two
// instruction mixes, below), and the final FMA is the one FP64 operation of
// the method.  A segment is 48 bytes in two arrays (one 256-bit and one
// 128-bit gather per element; the denser arrays also put more segments in a
// cache line).
#pragma once
#include <stdint.h>

namespace qm {
namespace fxt {

constexpr int K = 6;           // 64 segments in every binade
constexpr int E_LAST = 1072;   // binades e = -1 - E = 0 .. 1072 (x down to 2^-1073)
// rows (e + 1) 2^K + j: binade e = -1 (x = 1 exactly, u = 1/2) holds zero
// rows, which evaluate to z = +0
constexpr int N_ALL = (E_LAST + 2) << K;

// a0, B0 = b0 2^-s0, B1 = b1 2^-s0 (non-negative), and B2 = b2 2^-s0 in the
// low 52 bits with e0 = 1083 + s0 in the top 12
struct alignas(32) SegA {
    double a0;
    long long B0, B1, B2s;
};

// f_k = b_k 2^-s0, k = 3..6, rounded to single precision
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

// rn(G) for 0 <= G < 2^48, rounding to nearest even, exactly: the high half
// G div 2^24 by truncation, the low half G - 2^24 (G div 2^24) (exact in
// single precision, below 2^24) by rounding; the conversions are 32-bit ones.
__device__ __forceinline__ unsigned long long f32_to_u64_rn_split(float G)
{
    const unsigned gh = __float2uint_rz(G * 5.9604644775390625e-8f);            // G 2^-24, exact
    const float gl = __fmaf_rn(__uint2float_rz(gh), -16777216.0f, G);           // exact
    return (unsigned long long)gh * 16777216ull + __float2uint_rn(gl);
}

// Instruction mixes with bit-identical results, chosen per kernel by what
// bounds it: t_u as (1 + t_u) - 1, one exact FP64 add (FX_TU_FADD, the
// streaming kernel: FX_INT_LEAN), or by normalising Tu with integer
// operations (FX_FP64_LEAN, for kernels bound by FP64 maps: the final FMA is
// then the only FP64 instruction).
enum { FX_TU_FADD = 2, FX_INT_LEAN = 2, FX_FP64_LEAN = 0 };

// floor(a b / 2^64) for a < 2^62 and b < 2^63 from 32-bit limbs:
// a1 b1 + hi32(a0 b1 + a1 b0 + hi32(a0 b0)); the partial sums stay below 2^64,
// so this is the exact high half of the product.
__device__ __forceinline__ unsigned long long mulhi_q(unsigned long long a, unsigned long long b)
{
    const unsigned a0 = (unsigned)a, a1 = (unsigned)(a >> 32);
    const unsigned b0 = (unsigned)b, b1 = (unsigned)(b >> 32);
    const unsigned long long m1 = (unsigned long long)a1 * b0 + __umulhi(a0, b0);
    const unsigned long long m2 = (unsigned long long)a0 * b1 + m1;
    return (unsigned long long)a1 * b1 + (m2 >> 32);
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
    // e >= -1 for every bit pattern (x = 2d <= 1); the clamp keeps the index
    // inside the table whatever the input
    const int ec = min(max(e, -1), fxt::E_LAST) + 1;
    const unsigned j = (unsigned)(Mx >> sK) & ((1u << K) - 1u);
    const int idx = (ec << K) + (int)j;
    // offset back from the segment end, Tu = Tp + 1 in [1, 2^sK]: Tp is the
    // complement of the significand's low sK bits.  H is stored in the half
    // offset th = Tp 2^-(sK+1) in [0, 1/2) (re-expanded by one unit of the
    // offset), so th 2^64 is a plain shift below 2^63.
    const unsigned long long Tp = ~Mx & ((1ull << sK) - 1ull);
    const unsigned long long Tau = Tp << (11 + K);

    unsigned long long a0b, B0, B1, B2s;
    ld256(&T->a[idx], a0b, B0, B1, B2s);                           // a0, B0, B1, B2 | e0
    const float4 f = ld128f(&T->f[idx]);                            // f3..f6
    const unsigned long long B2 = B2s & ((1ull << 52) - 1ull);
    const unsigned e0 = (unsigned)(B2s >> 52);                      // 1083 + s0

    // single-precision tail from the top bits of the offset
    const float tf = __uint_as_float(0x4B000000u | (unsigned)(Tp >> 25)) - 8388608.0f;
    const float tau_f = tf * __uint_as_float((unsigned)(127 + K - 28) << 23);
    float F = __fmaf_rn(f.w, tau_f, f.z);
    F = __fmaf_rn(F, tau_f, f.y);
    F = __fmaf_rn(F, tau_f, f.x);
    // innermost step in single precision: th = Tp 2^-47 = hi 2^-24 + lo 2^-47
    // exactly (both halves are integers below 2^23),
    // F th = fl(fl(F 2^-24 hi) + F 2^-47 lo); acc = B2 + rn(F th)
    const float th = __uint_as_float(0x4B000000u | (unsigned)(Tp >> 23)) - 8388608.0f;
    const float tl = __uint_as_float(0x4B000000u | ((unsigned)Tp & 0x7FFFFFu)) - 8388608.0f;
    const float f24 = F * 5.9604644775390625e-8f;                  // 2^-24, exact
    const float G = __fmaf_rn(f24 * 1.1920928955078125e-07f, tl, __fmul_rn(f24, th));
    unsigned long long acc = B2 + f32_to_u64_rn_split(G);
    acc = B1 + mulhi_q(acc, Tau);
    acc = B0 + mulhi_q(acc, Tau);                                   // H 2^-s0 (0 on the zero rows)

    // H as a double: acc is in [2^61, 2^63) (H varies by under 1.6 % across a
    // segment, and s0 puts H(0) 2^-s0 in [2^61, 2^62)), so its leading bit is
    // bit 61 or 62: round to 53 bits by one shift, then add the exponent field;
    // the significand's leading bit carries into the exponent (a round-up to
    // 2^53 carries one further, to the next power of two, exactly)
    const unsigned top = (unsigned)(acc >> 62);
    const unsigned long long hm = (acc + (256ull << top)) >> (9 + top);
    const unsigned long long hbits = hm + ((unsigned long long)(e0 + top) << 52);
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
    return (unsigned long long)__double_as_longlong(g);
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
