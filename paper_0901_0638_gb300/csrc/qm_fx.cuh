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
//     |z| = a0 + t_u H,   H = b0 + th (b1 + th (b2 + th C)) > 0,   b_k = beta_k 2^k,
//     C   = b3 + th (b4 + th (b5 + th b6))   (32-bit integers, scale per segment)
//
// The Horner steps for b0 and b1 run on unsigned 64-bit accumulators (below
// 2^62) times th as a Q0.64 integer (below 2^63): the high half of the
// 128-bit product comes from three 32 x 32 -> 64-bit products (the low-limb
// product, below one unit of the result, is left out, so a step can come out
// one unit of 2^s0 low; the generator emulates exactly this).  b3..b6 form an
// inner chain on 32-bit integers under a per-segment scale 2^c (three high
// products by th as a Q0.32 integer), which enters the b2 step as
// B2 + (C th) 2^(c-32) through one 32 x 32 -> 64-bit product and a shift of
// 32 - c.  The normalisation of x is integer arithmetic, H becomes a double by
// bit assembly and t_u exactly (two instruction mixes, below), and the final
// FMA is the one FP64 operation of the method.  A segment is 48 bytes in two
// arrays (one 256-bit and one 128-bit gather per element; the denser arrays
// also put more segments in a cache line).
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

// C_k = b_k 2^-(s0 + c), k = 3..6, rounded to integers below 2^32 (C6 below
// 2^27), and the join shift 32 - c (0 .. 31) in the top five bits of c6s
struct alignas(16) SegC {
    unsigned c3, c4, c5, c6s;
};

struct FxTable {
    SegA a[N_ALL];
    SegC c[N_ALL];
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
__device__ __forceinline__ uint4 ld128u(const void* p)
{
    uint4 v;
    asm("ld.global.nc.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
    return v;
}

// Instruction mixes with bit-identical results, chosen per kernel by what
// bounds it: t_u as (1 + t_u) - 1, one exact FP64 add (FX_TU_FADD, the
// streaming kernel: FX_INT_LEAN), or by normalising Tu with integer
// operations (FX_FP64_LEAN, for kernels bound by FP64 maps: the final FMA is
// then the only FP64 instruction).
enum { FX_TU_FADD = 2, FX_INT_LEAN = 2, FX_FP64_LEAN = 0 };

// floor(a b / 2^64), or one less, for a < 2^62 and b < 2^63, from three of
// the four 32 x 32 -> 64-bit limb products: a1 b1 + hi32(a0 b1 + a1 b0).  The
// middle sum stays below 2^64 (a1 b0 < 2^62, a0 b1 < 2^63); leaving out
// hi32(a0 b0) < 2^32 lowers it by less than 2^32, so the result by at most 1.
__device__ __forceinline__ unsigned long long mulhi_q(unsigned long long a, unsigned long long b)
{
    const unsigned a0 = (unsigned)a, a1 = (unsigned)(a >> 32);
    const unsigned b0 = (unsigned)b, b1 = (unsigned)(b >> 32);
    const unsigned long long m = (unsigned long long)a0 * b1 + (unsigned long long)a1 * b0;
    return (unsigned long long)a1 * b1 + (m >> 32);
}

// The inner chain: C = C3 + th (C4 + th (C5 + th C6)) on 32-bit integers,
// th32 = floor(th 2^32) < 2^31 (each step's high product truncates), then
// floor(C th32 / 2^sh), sh = 32 - c, in the units 2^s0 of the outer chain.
// With ESTRIN the same polynomial as (C3 + th C4) + th^2 (C5 + th C6), th^2
// as hi32(th32 th32): two independent high products, then one (a shorter
// dependent chain; it truncates differently, within the same bounds).
template <bool ESTRIN = false>
__device__ __forceinline__ unsigned long long fx_inner(uint4 c, unsigned th32)
{
    unsigned a;
    if (ESTRIN) {
        const unsigned lo = __umulhi(c.y, th32) + c.x;
        const unsigned hi = __umulhi(c.w & 0x07FFFFFFu, th32) + c.z;
        a = __umulhi(hi, __umulhi(th32, th32)) + lo;
    } else {
        a = __umulhi(c.w & 0x07FFFFFFu, th32) + c.z;
        a = __umulhi(a, th32) + c.y;
        a = __umulhi(a, th32) + c.x;
    }
    return ((unsigned long long)a * th32) >> (c.w >> 27);
}

// One row of the layout above at th = Tau 2^-64 in [0, 1/2) (Tau < 2^63):
// fma(tu, H(th), a0), tu the row's multiplier (the offset t_u, exact).  The
// inner chain takes th32 = Tau >> 32 (Horner, or Estrin with ESTRIN: the two
// truncate differently).  HB is the position of the leading bit of
// H(0) 2^-s0 (61 for the quantile's rows, e0 = 1083 + s0; rows whose
// polynomial grows faster keep B2 inside its 52-bit field with a lower one,
// e0 = 1022 + HB + s0).
template <bool ESTRIN = false, int HB = 61>
__device__ __forceinline__ double fx_row_core(const fxt::SegA* A, const fxt::SegC* C, unsigned long long Tau,
                                              double tu)
{
    static_assert(HB >= 54 && HB <= 61, "H(0) 2^-s0 between 2^54 and 2^62");
    unsigned long long a0b, B0, B1, B2s;
    ld256(A, a0b, B0, B1, B2s);                                     // a0, B0, B1, B2 | e0
    const uint4 c = ld128u(C);                                      // C3..C6 | sh
    const unsigned long long B2 = B2s & ((1ull << 52) - 1ull);
    const unsigned e0 = (unsigned)(B2s >> 52);                      // 1022 + HB + s0

    unsigned long long acc = B2 + fx_inner<ESTRIN>(c, (unsigned)(Tau >> 32));
    acc = B1 + mulhi_q(acc, Tau);
    acc = B0 + mulhi_q(acc, Tau);                                   // H 2^-s0 (0 on the zero rows)

    // H as a double: acc is in [2^HB, 2^(HB+2)) (H varies by under a factor 2
    // across a segment, and s0 puts H(0) 2^-s0 in [2^HB, 2^(HB+1))), so its
    // leading bit is bit HB or HB + 1: round to 53 bits by one shift, then
    // add the exponent field; the significand's leading bit carries into the
    // exponent (a round-up to 2^53 carries one further, to the next power of
    // two, exactly)
    const unsigned top = (unsigned)(acc >> (HB + 1));
    const unsigned long long hm = (acc + ((1ull << (HB - 53)) << top)) >> (HB - 52 + top);
    const unsigned long long hbits = hm + ((unsigned long long)(e0 + top) << 52);
    return __fma_rn(tu, __longlong_as_double((long long)hbits), __longlong_as_double((long long)a0b));
}

// A row at the offset Tp = Tu - 1 back from the segment end (the complement
// of the significand's low 52 - K bits): fma(+-t_u, H, a0), with -t_u when
// neg (rows that store z = a0 - t_u H, as the exponential -> normal map's).
template <int MIX = FX_INT_LEAN>
__device__ __forceinline__ double fx_row_fma(const fxt::SegA* A, const fxt::SegC* C, unsigned long long Tp,
                                             bool neg = false)
{
    constexpr int K = fxt::K;
    // H is stored in the half offset th = Tp 2^-(sK+1) in [0, 1/2) (re-expanded
    // by one unit of the offset), so th 2^64 is a plain shift below 2^63.
    const unsigned long long Tau = Tp << (11 + K);
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
    // the sign of t_u on its bits (no FP64 instruction)
    tu = __longlong_as_double(__double_as_longlong(tu) ^ (long long)((unsigned long long)neg << 63));
    return fx_row_core(A, C, Tau, tu);
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
    // complement of the significand's low sK bits
    const unsigned long long Tp = ~Mx & ((1ull << sK) - 1ull);
    return (unsigned long long)__double_as_longlong(fx_row_fma<MIX>(&T->a[idx], &T->c[idx], Tp));
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
