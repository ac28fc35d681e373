// qm_exp_map.cuh -- the exponential -> normal recycling map
// z = Phi^{-1}(1 - e^{-x}) (Sec. 2.3, Sec. 6) on given samples x, in the
// fixed-point row layout of the FIXED normal quantile (qm_fx.cuh; rows:
// qm_exp_fx_tables.h, generated by fit/gen_exp_fx_tables.py from the
// recycling-ODE expansions).
//
// Every 2^-26 <= x < 128 takes segment j (top 6 bits of the significand) of
// its binade, with the offset t_u back from the segment end read from the
// bits (t_u = (Tp + 1) 2^-52, Tp = the complement of the low 46 bits), the
// same two 64-bit Horner steps and 32-bit inner chain as the FIXED kernel,
// and one FP64 FMA:
//   below the segment that holds ln 2:  z = -(a0 + t_u H),
//   from it on:                         z = a0 - t_u H.
// The segment [0.6875, 0.6953125) holds ln 2, where z passes through 0: its
// row reads z = a0 - t_u H across it, and |x - ln 2| < 2^-12 keeps relative
// accuracy in v = x - ln 2 (ln 2 split hi/lo): z = v P(tau),
// tau = 8 (1/32 - v), one row of its own (the row form of qm_t_fx.h), taken
// by a branch (about 1 in 4000 Exp(1) samples).  Out of line, rarely taken:
// x < 2^-26 (u = x - x^2/2 through the normal table), x >= 128 (the
// deep-tail rational in v), and the edge values.
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

// x in (0, 2^-26) or x >= 128 (v >= 127)
static __device__ __noinline__ double exp_to_normal_rare(double x)
{
    const double v = __dadd_rn(__dadd_rn(x, -0.69314718055994528623), -2.3190468138462996154e-17);
    if (v >= 64.0) return probit_mag_exp_deep(v);
    const double u = __fma_rn(-0.5 * x, x, x);          // 1 - e^{-x} to double precision
    const double mag = f64_tbl_covers(u) ? probit_mag_f64_tbl(u) : probit_mag_exp_deep(-log(2.0 * u));
    return -mag;
}

// the centre segment: z = v P(tau), v = x - ln 2 (relative-accurate near 0),
// t = 1/32 - v, tau = 8 t
__device__ __forceinline__ double exp_to_normal_centre(double x)
{
    constexpr uint64_t kMant = 0x000fffffffffffffull;
    const double v = __dadd_rn(__dadd_rn(x, -0.69314718055994528623), -2.3190468138462996154e-17);
    const double t = __dadd_rn(0.03125, -v);
    const uint64_t tb = (uint64_t)__double_as_longlong(t);
    const uint64_t Mt = (tb & kMant) | (1ull << 52);
    const int st = (int)((tb >> 52) & 0x7ff) - 1023 + 15;           // t 2^67
    const uint64_t Sig = st >= 0 ? ((Mt << min(st, 63)) & 0x7fffffffffffffffull) : (st > -64 ? (Mt >> (-st)) : 0ull);
    return segtx_eval<false>(&efx::ROW_C, Sig, v);
}

template <int MIX = FX_INT_LEAN>
__device__ __forceinline__ double exp_to_normal_fx(double x)
{
    static_assert(efx::X_K == fxt::K, "the rows share the FIXED layout");
    constexpr int K = efx::X_K;
    const uint64_t xb = (uint64_t)__double_as_longlong(x);
    if (xb == 0 || xb >= 0x7ff0000000000000ull) return exp_to_normal_edge(x);
    if (xb < 0x3E50000000000000ull || xb >= 0x4060000000000000ull) return exp_to_normal_rare(x);   // 2^-26, 128
    // every lane runs the binade path, then the lanes with |x - ln 2| < 2^-12
    // (about 1 in 4000 Exp(1) samples) take the centre row: z = a0 - t_u H
    // passes through 0 in the segment of ln 2, and away from it the
    // cancellation costs under 2e-15 relative
    const int row = (((int)(xb >> 52) - 1023 - efx::X_EMIN) << K) + (int)((xb >> (52 - K)) & ((1u << K) - 1u));
    const uint64_t Tp = ~xb & ((1ull << (52 - K)) - 1ull);
    const bool pos = xb >= efx::POS_BITS;
    double r = fx_row_fma<MIX>(efx::ROWS + row, efx::ROWS_IN + row, Tp, pos);
    r = __longlong_as_double(__double_as_longlong(r) ^ (long long)((unsigned long long)!pos << 63));
    if (xb - efx::NEAR_LO_BITS < efx::NEAR_HI_BITS - efx::NEAR_LO_BITS) r = exp_to_normal_centre(x);
    return r;
}

}  // namespace qm
