// qm_exp_map.cuh -- the exponential -> normal recycling map
// z = Phi^{-1}(1 - e^{-x}) (Sec. 2.3, Sec. 6) on given samples x, in the
// fixed-point row form of qm_t_fx.h (rows: qm_exp_fx_tables.h, generated by
// fit/gen_exp_fx_tables.py from the recycling-ODE expansions).
//
// Every lane takes one path; the region only selects a row, the offset tau and
// the multiplier of the final FMA (v = x - ln 2, relative-accurate near 0):
//   v >= 1/32:              |z| = a0 - t P(tau),  t = v_e - v (exact), v_e the segment end;
//   -1/64 <= v < 1/32:      z = v P(tau),         t = 1/32 - v (through 0 at x = ln 2);
//   2^-26 <= x < ln2 - 1/64: z = -(a0 + t_u P(tau)), t_u the offset of x's
//                           significand back from its segment end (binades
//                           of x, 32 segments each), read from the bits.
// Out of line, rarely taken: x < 2^-26 (u = x - x^2/2 through the normal
// table), v >= 64 (the deep-tail rational), and the edge values.
// Include in the translation units that use it (tables are per unit).
#pragma once

#include "qm_device.cuh"
#include "qm_exp_fx_tables.h"

namespace qm {

static __device__ __noinline__ double exp_to_normal_edge(double x)
{
    if (x == 0.0) return __longlong_as_double(0xfff0000000000000ll);      // -inf (also -0)
    if (x == __longlong_as_double(0x7ff0000000000000ll)) return x;          // +inf
    return __longlong_as_double(0x7ff8000000000000ll);                     // x < 0, NaN
}

// x in (0, 2^-26) (then v < 0) or v >= 64
static __device__ __noinline__ double exp_to_normal_rare(double x, double v)
{
    if (v >= 64.0) return probit_mag_exp_deep(v);
    const double u = __fma_rn(-0.5 * x, x, x);          // 1 - e^{-x} to double precision
    const double mag = f64_tbl_covers(u) ? probit_mag_f64_tbl(u) : probit_mag_exp_deep(-log(2.0 * u));
    return -mag;
}

__device__ __forceinline__ double exp_to_normal_fx(double x)
{
    constexpr uint64_t kMant = 0x000fffffffffffffull;
    const uint64_t xb = (uint64_t)__double_as_longlong(x);
    if (xb == 0 || xb >= 0x7ff0000000000000ull) return exp_to_normal_edge(x);
    const double kLn2Hi = 0.69314718055994528623, kLn2Lo = 2.3190468138462996154e-17;
    const double v = __dadd_rn(__dadd_rn(x, -kLn2Hi), -kLn2Lo);
    // the region tests on the bits of v (integer compares; FP64 compares
    // would issue on the FP64 pipe): v >= -1/64, v < 64, v < 1, v < 1/32
    const uint64_t vb = (uint64_t)__double_as_longlong(v);
    const bool vneg = (vb >> 63) != 0;
    const uint64_t vmag = vb & 0x7fffffffffffffffull;
    const bool vside = !vneg || vmag <= 0x3F90000000000000ull;                     // |v| <= 2^-6
    if (vside ? (!vneg && vmag >= 0x4050000000000000ull) : xb < 0x3E50000000000000ull)
        return exp_to_normal_rare(x, v);

    // V rows: v in [1/32, 1) width 1/32 (tau = 8 t), [1, 64) width 1/8
    // (tau = 2 t); row 0 for v < 1/32 (tau = 8 t)
    const int Ev = (int)((vb >> 52) & 0x7ff) - 1023;
    const uint64_t Mv = (vb & kMant) | (1ull << 52);
    const bool fine = vneg || vmag < 0x3FF0000000000000ull;                        // v < 1
    const bool row0 = vneg || vmag < 0x3FA0000000000000ull;                        // v < 1/32
    const int shv = min(max(fine ? 47 - Ev : 49 - Ev, 0), 63);
    const uint32_t q = (uint32_t)(Mv >> shv);                       // floor(32 v) or floor(8 v)
    const int rv = row0 ? 0 : min(fine ? (int)q : efx::V_FINE + (int)q - efx::V_COARSE, efx::NV - 1);
    const uint32_t nq = row0 ? 1u : (q + 1u) & 0xffffu;             // segment end nq 2^-p
    const int ln = 31 - __clz(nq | 1u);
    const uint64_t veb = ((uint64_t)(ln - (fine ? 5 : 3) + 1023) << 52) | (((uint64_t)nq << (52 - ln)) & kMant);

    // X rows: binade E = -1 .. -26 of x, segment j = top 5 bits of the
    // significand, Tp = complement of its low 47 bits (t_u = (Tp + 1) 2^-52)
    const int Ex = (int)(xb >> 52) - 1023;
    const int rx = (min(max(-1 - Ex, 0), (efx::NX >> efx::X_K) - 1) << efx::X_K) + (int)((xb >> 47) & 31u);
    const uint64_t Tp = ~xb & ((1ull << 47) - 1ull);

    // one exact subtraction serves the side taken: t = v_e - v, or
    // t_u = (1 + t_u) - 1
    const double d = __dadd_rn(__longlong_as_double((long long)(vside ? veb : 0x3FF0000000000001ull + Tp)),
                               vside ? -v : -1.0);
    const uint64_t tb = (uint64_t)__double_as_longlong(d);
    const uint64_t Mt = (tb & kMant) | (1ull << 52);
    const int st = (int)((tb >> 52) & 0x7ff) - 1023 + 12 + (fine ? 3 : 1);   // t 2^(64 + k)
    const uint64_t SigV = (tb == 0) ? 0ull
                        : (st >= 0 ? ((Mt << min(st, 63)) & 0x7fffffffffffffffull)
                                   : (st > -64 ? (Mt >> (-st)) : 0ull));

    const ttbl::SegTX* row = vside ? (efx::ROWS_V + rv) : (efx::ROWS_X + rx);
    const double r = segtx_eval<false>(row, vside ? SigV : (Tp << 16), vside ? (row0 ? v : -d) : d);
    return vside ? r : -r;
}

}  // namespace qm
