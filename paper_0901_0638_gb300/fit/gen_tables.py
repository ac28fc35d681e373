"""Generate csrc/qm_tables.h: segment tables of the table-driven normal quantile.

The quantile is evaluated in the paper's exponential coordinate
v = -log(2d), d = min(u, 1-u) (Sec. 6), but the logarithm is never formed.
Write x = 2d = 2^E m with m in [1, 2); the top k bits of m pick a segment j
with a short reduction constant c_j ~ 1/(segment centre) (c = 1/2 for the top
segment, which makes r exact at the centre of the distribution), and

    r = m c_j - 1,       v = V_{E,j} - log(1 + r),  V_{E,j} = -E ln2 + ln c_j.

Around V the function Q(v) = Phi^{-1}(1 - e^{-v}/2) is expanded with the
recycling ODE of the exponential background, Q'' + Q' = Q Q'^2 (Sec. 2.3,
Sec. 6; rode.taylor_exp_background), and composed with -log(1 + r), giving
per segment the Taylor coefficients of G(r) = Q(V - log(1 + r)).  A kernel
evaluates |Phi^{-1}(u)| = G(r) with a short Horner chain: no logarithm, no
division.

FP64 table: E = -1 .. -64 (v <= 44.4), k = 6 (64 segments per binade);
  entry = a0..a3, c (double) | a4..a7 (float)           -- 64 bytes.
  (a0..a3 are evaluated in double, a4..a7 in single precision: with 64
  segments per binade their terms are below 3e-9, 5e-10 and 2e-14 of the
  result, so single precision adds at most ~1e-16.)
FP64 deep table (qm_tables_deep.h, used by the streaming FP64 kernel only):
  E = -65 .. -1022 (x = 2d normal, 44.4 < v <= 708), k = 5, same entry
  layout and degree (their single-precision terms are below 2e-10).
FP32 table: E = -1 .. -149, k = 5 (32 segments per binade), with the
  subtractive reduction r = m - m_j (m_j the segment centre, or 2 for the top
  segment, where r = 2x - 2 is exact and G(0) = 0 at u = 1/2), so
  G(r) = Q(V - log(1 + r/m_j)), V = -E ln2 - ln m_j;
  entry = a0..a3 (float)                                 -- 16 bytes, one load.
Usage:  python -m paper_0901_0638_gb300.fit.gen_tables
"""
from __future__ import annotations

import multiprocessing as mproc
import os
import sys

import mpmath as mp
import numpy as np

from . import rode
from . import targets as T

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(os.path.dirname(HERE), "csrc", "qm_tables.h")
OUT_DEEP = os.path.join(os.path.dirname(HERE), "csrc", "qm_tables_deep.h")
DEEP_K, DEEP_EHI, DEEP_ELO = 5, -65, -1022

F64_K, F64_EMIN, F64_DEG = 6, -64, 7
F32_K, F32_EMIN, F32_DEG = 5, -149, 3


def seg_const(j, k):
    if j == 2**k - 1:
        return 0.5
    lo = 1.0 + j / 2.0**k
    hi = 1.0 + (j + 1) / 2.0**k
    c = 2.0 / (lo + hi)
    return float(np.float32(float(np.float32(c))))  # a float, exact in double


def seg_coeffs(args):
    E, j, k, deg = args
    mp.mp.dps = 45
    c = mp.mpf(seg_const(j, k))
    V = -E * mp.log(2) + mp.log(c)
    if E == -1 and j == 2**k - 1:
        V = mp.mpf(0)
        q0, q1 = mp.mpf(0), mp.sqrt(mp.pi / 2)
    else:
        q0 = T.q_exp(V)
        q1 = mp.exp(-V) / 2 / mp.npdf(q0)      # Q' = (e^{-v}/2) / phi(Q)
    b = rode.taylor_exp_background(V, q0, q1, deg + 2)
    a = rode.compose(b, rode.neg_log1p_series(deg + 2), deg + 2)
    # check: evaluate the truncated, rounded polynomial at the segment ends
    mlo = 1 + mp.mpf(j) / 2**k
    mhi = 1 + mp.mpf(j + 1) / 2**k
    worst = mp.mpf(0)
    for m in (mlo, (mlo + mhi) / 2, mhi - mp.mpf(2) ** -40):
        r = m * c - 1
        x = m * mp.mpf(2) ** E
        ref = T.q_exp(-mp.log(x)) if x != 1 else mp.mpf(0)
        approx = sum(a[n] * r**n for n in range(deg + 1))
        if ref != 0:
            worst = max(worst, abs(approx / ref - 1))
    return (E, j, float(c), [a[n] for n in range(deg + 1)], float(worst))


def seg_coeffs_sub(args):
    """FP32 segments: subtractive reduction r = m - m_j."""
    E, j, k, deg = args
    mp.mp.dps = 45
    top = j == 2**k - 1
    mj = mp.mpf(2) if top else 1 + (mp.mpf(j) + mp.mpf("0.5")) / 2**k
    V = -E * mp.log(2) - mp.log(mj)
    if E == -1 and top:
        V = mp.mpf(0)
        q0, q1 = mp.mpf(0), mp.sqrt(mp.pi / 2)
    else:
        q0 = T.q_exp(V)
        q1 = mp.exp(-V) / 2 / mp.npdf(q0)
    b = rode.taylor_exp_background(V, q0, q1, deg + 2)
    s = [mp.mpf(0)] + [mp.mpf((-1) ** n) / n / mj**n for n in range(1, deg + 3)]  # -log(1 + r/mj)
    a = rode.compose(b, s, deg + 2)
    mlo = 1 + mp.mpf(j) / 2**k
    mhi = 1 + mp.mpf(j + 1) / 2**k
    worst = mp.mpf(0)
    for m in (mlo, (mlo + mhi) / 2, mhi - mp.mpf(2) ** -30):
        r = m - mj
        x = m * mp.mpf(2) ** E
        ref = T.q_exp(-mp.log(x)) if x != 1 else mp.mpf(0)
        approx = sum(a[n] * r**n for n in range(deg + 1))
        if ref != 0:
            worst = max(worst, abs(approx / ref - 1))
    return (E, j, float(mj), [a[n] for n in range(deg + 1)], float(worst))


def hexd(x):
    return float(x).hex()


def hexf(x):
    return float(np.float32(float(x))).hex() + "f"


def main():
    jobs64 = [(E, j, F64_K, F64_DEG) for E in range(-1, F64_EMIN - 1, -1) for j in range(2**F64_K)]
    jobs32 = [(E, j, F32_K, F32_DEG) for E in range(-1, F32_EMIN - 1, -1) for j in range(2**F32_K)]
    jobsd = [(E, j, DEEP_K, F64_DEG) for E in range(DEEP_EHI, DEEP_ELO - 1, -1) for j in range(2**DEEP_K)]
    with mproc.Pool(max(1, (os.cpu_count() or 2))) as pool:
        r64 = pool.map(seg_coeffs, jobs64, chunksize=16)
        r32 = pool.map(seg_coeffs_sub, jobs32, chunksize=16)
        rd = pool.map(seg_coeffs, jobsd, chunksize=32)
    wd = max(r[4] for r in rd)
    print(f"FP64 deep table: {len(rd)} segments, truncation <= {wd:.3g}", file=sys.stderr)
    dl = [
        "// Generated by paper_0901_0638_gb300/fit/gen_tables.py -- do not edit.\n",
        "// Deep-tail extension of the FP64 segment table (same entry layout):\n",
        f"// E = {DEEP_EHI}..{DEEP_ELO}, k = {DEEP_K}, degree {F64_DEG}, max truncation {wd:.3g}.\n",
        "// Index (-65 - E) 2^k + j.  Include in one translation unit only.\n",
        "#pragma once\n#include \"qm_tables.h\"\n\nnamespace qm {\nnamespace tbl {\n\n",
        f"constexpr int DEEP_K = {DEEP_K};\nconstexpr int DEEP_EHI = {DEEP_EHI};\nconstexpr int DEEP_ELO = {DEEP_ELO};\n\n",
        f"__device__ const SegF64 SEG_F64_DEEP[{len(rd)}] = {{\n",
    ]
    for E, j, c, a, _ in rd:
        dl.append("  {{" + ",".join(hexd(x) for x in a[:4]) + "}," + hexd(c) + ",{" +
                  ",".join(hexf(x) for x in a[4:8]) + "},{0.0f,0.0f}},\n")
    dl.append("};\n\n}  // namespace tbl\n}  // namespace qm\n")
    with open(OUT_DEEP, "w") as f:
        f.write("".join(dl))
    w64 = max(r[4] for r in r64)
    w32 = max(r[4] for r in r32)
    print(f"FP64 table: {len(r64)} segments, truncation <= {w64:.3g}", file=sys.stderr)
    print(f"FP32 table: {len(r32)} segments, truncation <= {w32:.3g}", file=sys.stderr)
    lines = [
        "// Generated by paper_0901_0638_gb300/fit/gen_tables.py -- do not edit.\n",
        "// Segment tables of the table-driven normal quantile: per segment (E, j)\n",
        "// of x = 2d = 2^E m, the Taylor coefficients in r = m c - 1 of\n",
        "// G(r) = Q(V - log(1+r)), Q the exponential-coordinate normal quantile,\n",
        "// obtained from the recycling ODE Q'' + Q' = Q Q'^2.  Index (-1-E) 2^k + j.\n",
        f"// FP64: k = {F64_K}, E = -1..{F64_EMIN}, degree {F64_DEG}, max truncation {w64:.3g}.\n",
        f"// FP32: k = {F32_K}, E = -1..{F32_EMIN}, degree {F32_DEG}, max truncation {w32:.3g}.\n",
        "#pragma once\n\nnamespace qm {\nnamespace tbl {\n\n",
        f"constexpr int F64_K = {F64_K};\nconstexpr int F64_EMIN = {F64_EMIN};\n",
        f"constexpr int F32_K = {F32_K};\nconstexpr int F32_EMIN = {F32_EMIN};\n\n",
        "struct alignas(64) SegF64 { double a[4]; double c; float b[4]; float pad[2]; };\n",
        "struct alignas(16) SegF32 { float a0, a1, a2, a3; };\n\n",
        f"__device__ const SegF64 SEG_F64[{len(r64)}] = {{\n",
    ]
    for E, j, c, a, _ in r64:
        lines.append("  {{" + ",".join(hexd(x) for x in a[:4]) + "}," + hexd(c) + ",{" +
                     ",".join(hexf(x) for x in a[4:8]) + "},{0.0f,0.0f}},\n")
    lines.append("};\n\n")
    lines.append(f"__device__ const SegF32 SEG_F32[{len(r32)}] = {{\n")
    for E, j, c, a, _ in r32:
        lines.append("  {" + ",".join(hexf(x) for x in a[:4]) + "},\n")
    lines.append("};\n\n}  // namespace tbl\n}  // namespace qm\n")
    with open(OUT, "w") as f:
        f.write("".join(lines))
    print("wrote", OUT, file=sys.stderr)


if __name__ == "__main__":
    main()
