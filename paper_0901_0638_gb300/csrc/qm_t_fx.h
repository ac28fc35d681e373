// qm_t_fx.h -- layout of the Student-t segment rows as the device evaluates
// them: the normal -> t_nu recycling map (Sec. 3) in 64-bit fixed point with
// one FP64 FMA per element.
//
// The host tables (offline fits for the tabulated nu, or tables built at run
// time for any other nu) hold, per segment j of width 1/32 on 0 <= |z| < 8.75,
// the coefficients c_0..c_9 of the expansion in s = |z| - (j + 1/2)/32 (in
// s = |z| for j = 0, the central series).  Before upload every segment is
// re-expanded about its start z_j = j/32 (sigma = |z| - z_j in [0, 1/32);
// z_0 = 0): on every segment of every nu these coefficients are non-negative
// (the map is absolutely monotone on z > 0; checked at conversion), so
//
//     |t| = a0 + sigma P,   P = sum_k d_k tau^k,   tau = 16 sigma in [0, 1/2),
//
// with d_k = c'_{k+1} 16^-k >= 0, runs on unsigned integers: d_0..d_4 as
// integers D_k = d_k 2^-s0 (s0 puts D_0 in [2^59, 2^60], which keeps D_4
// below 2^52 beside the exponent field; P varies by less than a factor 2
// across a segment, so the accumulator stays in [2^59, 2^61)), a
// Horner chain acc = D_k + mulhi(acc, tau 2^64) (the high half of the 128-bit
// product from three 32-bit limb products: exact or one unit low), and
// d_5..d_8 as an inner chain on 32-bit integers C_k = d_k 2^-(s0 + c) under
// a per-segment scale 2^c, in tau32 = floor(tau 2^32): a = C_5 + hi32(tau32
// (C_6 + ...)), every partial value below 2^32, which enters the d_4 step as
// D_4 + floor(a tau32 / 2^(32 - c)); the shift 32 - c (0 .. 31) sits in the
// top five bits of the C_8 word (C_8 below 2^27).  The d_5 term is at most
// ~4e-6 of |t| (nu = 0.75 at |z| = 8.75), so the 32-bit chain costs it under
// 1e-15.  P becomes a double by one rounding shift and the exponent field
// e0 = 1081 + s0, and |t| = fma(sigma, P, a0) is the one FP64 operation
// besides the exact sigma = |z| - z_j.
#pragma once
#include <stdint.h>

#include "qm.h"

namespace qm {
namespace ttbl {

struct alignas(64) SegTX {
    double a0;                      // |t| at the segment start
    unsigned long long D0, D1, D2;  // d_0..d_2 2^-s0
    unsigned long long D3;          // d_3 2^-s0
    unsigned long long D4e;         // d_4 2^-s0 (below 2^52) | e0 << 52
    unsigned c[4];                  // C_5, C_6, C_7, C_8 | (32 - c) << 27
};
static_assert(sizeof(SegTX) == 64, "one 64-byte row per segment");

}  // namespace ttbl

// Converts nseg segment rows of coefficients c_0..c_9 (seg10[10 j + k],
// expansion about the segment centre (j + 1/2)/32, about 0 for j = 0) into
// the fixed-point rows above.  Checks the sign, range and accuracy conditions
// (the conversion is re-evaluated at points of every segment against the
// original polynomial, within 1e-13 relative); QM_ERR_UNSUPPORTED if a
// segment violates one.
qm_status t_pack_fx(const double* seg10, int nseg, ttbl::SegTX* out);

// Rows for maps whose segment coefficients have mixed signs (the same 64-byte
// SegTX layout, read by segts_eval): Q(start + sigma) = a0 + sigma P(tau),
// tau = sigma / (2 w) in [0, 1/2) for a segment of width w, P > 0 but d_1..d_8
// of either sign.  The unsigned chain then runs on biased accumulators:
// acc_k + 2^60 for the outer steps (|acc_k| < 2^60; each step subtracts
// floor(Sig / 16) = floor(2^60 tau), the bias carried through the high
// product), D_1..D_3 stored as d_k 2^-s0 + 2^60, D_4 as d_4 2^-s0 + 2^51 in
// the low 52 bits of D4e; the 32-bit inner chain on a_k + 2^29 (|a_k| < 2^29,
// C_8 + 2^25 below 2^27 beside the shift).  s0 puts P 2^-s0 in [2^59, 2^61)
// over the whole segment (P varies by less than a factor 2; checked from
// the coefficient bounds), e0 = 1081 + s0.
//
// coef: c_0..c_9 of Q in s = sigma - h about the point h from the segment
// start (h = w / 2 for the centre; h = 0 keeps a0 = c_0 exactly).  Checks the
// ranges and the packed form against the original polynomial at points of
// the segment (relative 1e-13); QM_ERR_UNSUPPORTED if one fails.
qm_status pack_fx_biased(const double* coef, double w, double h, ttbl::SegTX* out);

}  // namespace qm
