// qm_t_fx.h -- layout of the fixed-point segment rows the device evaluates
// with one FP64 FMA: the Student-t rows of the normal -> t_nu recycling map
// (Sec. 3), and the 64-byte rows of the maps read by segtx_eval/segts_eval.
//
// Student t (TRows).  The host tables (offline fits for the tabulated nu, or
// tables built at run time for any other nu) hold, per segment j of width
// 1/32 on 0 <= |z| < 8.75, the coefficients c_0..c_9 of the expansion in
// s = |z| - (j + 1/2)/32 (in s = |z| for j = 0, the central series).  Before
// upload every segment is split into four rows of width 1/128, each
// re-expanded about its start z_r = r/128 (sigma = |z| - z_r in [0, 1/128))
// and truncated to degree 7 (under 2e-13 relative at nu = 0.75, the heaviest
// tail; checked at conversion).  On every row of every nu these coefficients
// are non-negative (the map is absolutely monotone on z > 0; checked), so
// each row is stored in the layout of the FIXED normal quantile (qm_fx.cuh):
//
//     |t| = a0 + sigma H(th),   th = 64 sigma in [0, 1/2),
//
// H = sum b'_k th^k with b'_0..b'_2 as integers B_k = b'_k 2^-s0 (s0 puts
// H(0) 2^-s0 in [2^58, 2^59), three bits lower than the quantile's rows, so
// that B_2 fits its 52-bit field for the heaviest tail: b'_2 reaches 2^-7.4
// b'_0 at nu = 0.75; H varies by less than a factor 2 over a row)
// and b'_3..b'_6 as 32-bit integers under a per-row scale (the inner chain),
// evaluated by fx_row_core: two Horner steps with high products from three
// 32-bit limb products, H to a double by bit assembly, |t| = fma(sigma, H,
// a0) the one FP64 operation besides the exact sigma.
//
// SegTX (64 bytes, the exponential -> normal centre row, the hyperbolic and
// t-copula rows): P = sum d_k tau^k, d_0..d_4 as integers D_k = d_k 2^-s0 (s0
// puts D_0 in [2^59, 2^60], which keeps D_4 below 2^52 beside the exponent
// field e0 = 1081 + s0), a Horner chain acc = D_k + mulhi(acc, tau 2^64), and
// d_5..d_8 as an inner chain on 32-bit integers C_k = d_k 2^-(s0 + c) under a
// per-segment scale 2^c, which enters the d_4 step as D_4 + floor(a tau32 /
// 2^(32 - c)); the shift 32 - c (0 .. 31) sits in the top five bits of the
// C_8 word (C_8 below 2^27).  P becomes a double by one rounding shift and
// the exponent field, and the row's value is fma(mlt, P, a0).
#pragma once
#include <stdint.h>

#include "qm.h"
#include "qm_fx.cuh"

namespace qm {
namespace ttbl {

// The Student-t rows of one nu: rows r = 0 .. T_NROW - 1 cover
// [r/128, (r+1)/128) of 0 <= |z| < 8.75, in the FIXED layout (two arrays:
// a 256-bit and a 128-bit gather per element).
constexpr int T_ROWS_PER_UNIT = 128;
constexpr int T_NROW = 1120;                // 8.75 x 128
constexpr int T_HB = 58;                    // H(0) 2^-s0 in [2^58, 2^59), e0 = 1080 + s0
struct TRows {
    fxt::SegA a[T_NROW];
    fxt::SegC c[T_NROW];
};

struct alignas(64) SegTX {
    double a0;                      // |t| at the segment start
    unsigned long long D0, D1, D2;  // d_0..d_2 2^-s0
    unsigned long long D3;          // d_3 2^-s0
    unsigned long long D4e;         // d_4 2^-s0 (below 2^52) | e0 << 52
    unsigned c[4];                  // C_5, C_6, C_7, C_8 | (32 - c) << 27
};
static_assert(sizeof(SegTX) == 64, "one 64-byte row per segment");

}  // namespace ttbl

// Converts the nseg = T_NROW / 4 Student-t segments of coefficients c_0..c_9
// (seg10[10 j + k], expansion about the segment centre (j + 1/2)/32, about 0
// for j = 0) into the TRows above: four rows per segment.  Checks the sign,
// range and accuracy conditions (every row re-evaluated at points of the row
// against the original polynomial, within 1e-12 relative: the degree-7
// truncation stays below 2e-13 for nu >= 0.75); QM_ERR_UNSUPPORTED if a row
// violates one.
qm_status t_pack_rows(const double* seg10, int nseg, ttbl::TRows* out);

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
