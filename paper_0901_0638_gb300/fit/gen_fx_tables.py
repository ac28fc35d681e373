"""Generate csrc/qm_fx_tables.h: the FP64 normal-quantile segment table for
evaluation in 64-bit fixed point.

The expansion is the one of gen_tables.py, in the paper's exponential
coordinate v = -log(2d), d = min(u, 1-u) (Sec. 6): x = 2d = 2^E m with
m in [1, 2); the top K bits of m select a segment of width 2^-K.  Around the
segment centre m_c (m_c = 2 on the top segment of the top binade, where z = 0
at x = 1) the recycling ODE of the exponential background,
Q'' + Q' = Q Q'^2 (Sec. 2.3, Sec. 6), gives the Taylor coefficients of

    |Phi^{-1}(u)| = G(t) = Q(V - log(1 + t/m_c)),  t = m - m_c,
    V = -E ln2 - ln m_c.

The kernel evaluates G in the unsigned offset t_u = m_end - m > 0 from the
segment's end m_end (x = 1 on the top segment, where G is odd in t and
z -> 0 keeps full relative accuracy).  The polynomial is the centre expansion
re-expanded about the end (the same polynomial, so the same truncation
error); |z| grows away from the end, so H > 0 on every segment:

    G = a_0 + t_u H(t_u),  H = sum_{k=0}^{6} beta_k tau^k,
    tau = t_u 2^K in (0, 1].

With the integer offset Tu = t_u 2^52 in [1, 2^(52-K)], the kernel reads
Tu - 1 = ~m & (2^(52-K) - 1) straight from the significand bits, so H is
stored re-expanded in tau' = tau - 2^(K-52) = (Tu - 1) 2^(K-52) in
[0, 1 - 2^(K-52)] (an exact change of expansion point, so the same
polynomial): tau' 2^64 = (Tu - 1) << (12 + K) always fits 64 bits.

Every coefficient beta_k is positive on every segment (asserted below): the
tail quantile |Phi^{-1}| as a function of the offset back from the segment
end has all its derivatives positive, so every Horner accumulator is
non-negative and the chain runs on unsigned integers.

On GB300 the FP64 pipe issues about 1/62 of the FP32 rate, so the
polynomial runs on the integer pipes, in the half offset th = tau'/2 in
[0, 1/2) on the coefficients beta'_k = beta_k 2^k (the same polynomial in
th).  beta'_0..beta'_2 are applied by a Horner chain on 64-bit unsigned
integers, th an unsigned Q0.64 number below 2^63:
acc_k = B_k + mulhi(acc_{k+1}, th 2^64), every acc in units of 2^s0 and
below 2^62.  mulhi is the high half of the 128-bit product formed from three
32 x 32 -> 64-bit limb products, a1 b1 + hi32(a0 b1 + a1 b0) (the middle sum
stays below 2^64): the exact high half or one less, emulated here exactly.
beta'_3..beta'_6 form an inner chain on 32-bit integers
C_k = beta'_k 2^-(s0 + c) under a per-segment scale 2^c, with th as a Q0.32
number th32 = floor(th 2^32) < 2^31: a = C3 + hi32(th32 (C4 + hi32(th32
(C5 + hi32(th32 C6))))), kept below 2^32 by the choice of c (asserted), and it
enters as acc_2 = B_2 + floor(a th32 / 2^(32 - c)).  The join shift 32 - c
(0 .. 31) sits in the top five bits of the C6 word (C6 < 2^27, asserted).
s0 puts H(0) 2^-s0 in [2^61, 2^62), and H
varies by less than a factor 2 across a segment (asserted; at most 1.6 %), so
acc_0 lies in [2^61, 2^63): its leading bit is bit 61 or 62, and H becomes a
double by one rounding shift and one add of the exponent field
(e0 + top) << 52, e0 = 1083 + s0 stored per segment, the significand's
implicit bit carrying into the exponent.  Then z = fma(t_u, H, a_0), with
t_u = (1 + t_u) - 1 formed exactly by one double-precision add.

Binades: e = -1 - E in [0, 1072], 64 segments each (K = 6), so every
double 0 < u < 1 (subnormal u included: x is normalised as an integer)
falls in a segment.  The table starts with 64 zero rows for e = -1, i.e.
x = 1 exactly (u = 1/2): a0 = 0 and H = +0 there (an all-zero accumulator
with a zero exponent field assembles to +0), so z = +0 needs no branch.

Entry: two arrays, so that a lane gathers 48 bytes with one 256-bit and one
128-bit load: A[i] = {a0 (double), B0, B1 (uint64), B2 | e0 << 52} (32 bytes;
B2 in the low 52 bits, e0 in the top 12) and
C[i] = {C3, C4, C5, C6 | (32 - c) << 27} (uint32, 16 bytes).

The generator checks every segment by emulating the kernel's integer and
double-precision steps exactly at both ends and interior points of the
segment, against the mpmath quantile, and prints the worst relative error.
Usage:  python -m paper_0901_0638_gb300.fit.gen_fx_tables
"""
from __future__ import annotations

import math
import multiprocessing as mproc
import os
import sys
from fractions import Fraction

import mpmath as mp
import numpy as np

from . import rode
from . import targets as T

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(os.path.dirname(HERE), "csrc", "qm_fx_tables.h")

DEG = 7                 # a_0..a_7
NI = 3                  # beta_0..beta_2 in fixed point
K_MAIN, E_MAIN = 6, 64  # binade index e = -1 - E in [0, 64): K = 6
K_DEEP, E_LAST = 6, 1072  # e in [64, 1072]: K = 6 too (x down to 2^-1073); one K
                          # everywhere makes every shift of the kernel a constant
N_MAIN = E_MAIN << K_MAIN
N_ALL = N_MAIN + ((E_LAST - E_MAIN + 1) << K_DEEP)


def seg_k(e):
    return K_MAIN if e < E_MAIN else K_DEEP


def seg_index(e, j):
    return (e << K_MAIN) + j if e < E_MAIN else N_MAIN + ((e - E_MAIN) << K_DEEP) + j


def is_top(e, j, K):
    return e == 0 and j == 2**K - 1


def centre_int(e, j, K):
    """Integer segment centre M_c of the 53-bit significand M of x."""
    if is_top(e, j, K):
        return 2**53
    return 2**52 + j * 2**(52 - K) + 2**(51 - K)


def taylor(e, j, K):
    """Coefficients of G about the anchor, in t_u (see the module docstring)."""
    mp.mp.dps = 50
    E = -1 - e
    top = is_top(e, j, K)
    mc = mp.mpf(centre_int(e, j, K)) / 2**52
    if top:
        V = mp.mpf(0)
        q0, q1 = mp.mpf(0), mp.sqrt(mp.pi / 2)
    else:
        V = -E * mp.log(2) - mp.log(mc)
        q0 = T.q_exp(V)
        q1 = mp.exp(-V) / 2 / mp.npdf(q0)   # Q' = (e^{-v}/2) / phi(Q)
    b = rode.taylor_exp_background(V, q0, q1, DEG + 2)
    s = [mp.mpf(0)] + [mp.mpf((-1) ** n) / n / mc**n for n in range(1, DEG + 3)]   # -log(1 + t/mc)
    a = rode.compose(b, s, DEG + 2)[:DEG + 1]
    h2 = mp.mpf(0) if top else mp.mpf(2) ** (-K - 1)              # t = h2 - t_u
    g = [mp.mpf(0)] * (DEG + 1)
    for k in range(DEG + 1):
        for i in range(k + 1):
            g[i] += a[k] * mp.binomial(k, i) * h2 ** (k - i) * (-1) ** i
    return g


def shift_poly(beta, delta):
    """Coefficients in tau' of H(tau' + delta) (exact re-expansion)."""
    n = len(beta)
    return [sum(beta[i] * mp.binomial(i, k) * delta ** (i - k) for i in range(k, n)) for k in range(n)]


def quantise(e, j, K, g):
    beta = [g[k + 1] * mp.mpf(2) ** (-K * k) for k in range(DEG)]
    beta = shift_poly(beta, mp.mpf(2) ** (K - 52))             # argument tau' = tau - 2^(K-52)
    assert all(b > 0 for b in beta), (e, j)                       # unsigned fixed point
    bh = [beta[k] * mp.mpf(2) ** k for k in range(DEG)]           # argument th = tau'/2
    assert sum(beta) < 2 * beta[0], (e, j)                        # H(1/2) / H(0) < 2
    s0 = int(mp.floor(mp.log(beta[0], 2))) - 61                   # H(0) 2^-s0 in [2^61, 2^62)
    B = [int(mp.nint(bh[k] / mp.mpf(2) ** s0)) for k in range(NI)]
    e0 = 1083 + s0                                                # exponent field base (below)
    assert 0 < B[2] < 2**51 and 0 < e0 < 2**11, (e, j, B[2], s0)  # B2 | e0 << 52
    # inner chain: C_k = b'_k 2^-(s0 + c) on 32-bit integers; for th < 1/2
    # the Horner value after the C_k step stays below C_k + C_{k+1}/2 + ...,
    # and c keeps every one of these partial sums below 2^32
    fk = [bh[k] / mp.mpf(2) ** s0 for k in range(NI, DEG)]

    def partial_max(v):
        return max(sum(v[i] * mp.mpf(2) ** (k - i) for i in range(k, len(v))) for k in range(len(v)))

    c = max(1, int(mp.ceil(mp.log(partial_max(fk), 2))) - 32)
    while True:
        C = [int(mp.nint(x / mp.mpf(2) ** c)) for x in fk]
        if partial_max([mp.mpf(x) for x in C]) < 2**32 - 8:
            break
        c += 1
    assert 1 <= c <= 32 and C[-1] < 2**27, (e, j, c, C)         # join shift 32 - c in 0 .. 31
    return {"a0": float(g[0]), "B": B, "C": C, "sh": 32 - c, "s0": s0, "e0": e0}


def mulhi_limbs(a, b):
    """floor(a b / 2^64) as the kernel forms it from three 32-bit limb
    products (a < 2^62, b < 2^63): a1 b1 + hi32(a0 b1 + a1 b0), the middle sum
    below 2^64.  The exact high half or one less."""
    a0, a1, b0, b1 = a & 0xFFFFFFFF, a >> 32, b & 0xFFFFFFFF, b >> 32
    m = a0 * b1 + a1 * b0
    assert m < 2**64
    r = a1 * b1 + (m >> 32)
    assert 0 <= ((a * b) >> 64) - r <= 1
    return r


def inner(q, th32):
    """The kernel's 32-bit inner chain C3 + th (C4 + th (C5 + th C6)) and its
    join floor(C th32 / 2^sh) into the units of the outer chain."""
    C = q["C"]
    a = C[-1]
    for ck in reversed(C[:-1]):
        a = ck + ((a * th32) >> 32)
        assert a < 2**32
    return (a * th32) >> q["sh"]


def emulate(q, K, Tu):
    """The kernel's arithmetic for the integer offset Tu; returns the double z."""
    Tp = Tu - 1                                                   # the kernel's ~m & (2^(52-K) - 1)
    Tau = Tp << (11 + K)                                          # th 2^64 = tau' 2^63
    assert 0 <= Tau < 2**63
    acc = q["B"][NI - 1] + inner(q, Tp >> 15)                     # th32 = th 2^32 = Tp 2^-15
    assert acc < 2**62
    acc = q["B"][1] + mulhi_limbs(acc, Tau)
    assert acc < 2**62
    acc = q["B"][0] + mulhi_limbs(acc, Tau)
    assert 2**61 <= acc < 2**63                                   # leading bit 61 or 62
    top = acc >> 62
    mant = (acc + (256 << top)) >> (9 + top)                      # rounded 53-bit significand
    hd = float(Fraction(mant) * Fraction(2) ** (9 + top + q["s0"]))
    # the kernel's bit assembly: mant (implicit bit included) + (e0 + top) << 52
    bits = mant + ((q["e0"] + top) << 52)
    assert np.frombuffer(np.uint64(bits).tobytes(), dtype=np.float64)[0] == hd
    t = Fraction(Tu) * Fraction(2) ** -52
    return float(t * Fraction(hd) + Fraction(q["a0"]))


def truth(e, Mx):
    mp.mp.dps = 40
    x = mp.mpf(Mx) * mp.mpf(2) ** (-1 - e - 52)
    if x == 1:
        return mp.mpf(0)
    return T.upper_probit(x / 2)


def job(args):
    e, j = args
    K = seg_k(e)
    g = taylor(e, j, K)
    q = quantise(e, j, K, g)
    full = 2**(52 - K)
    if e < E_MAIN:
        pts = [1, 2, 3, full // 3, full // 2, full - 1, full]
    else:
        pts = [1, full // 2, full]
    worst = 0.0
    for Tu in pts:
        z = emulate(q, K, Tu)
        Mx = 2**52 + (j + 1) * full - Tu
        w = truth(e, Mx)
        if w != 0:
            worst = max(worst, float(abs(mp.mpf(z) / w - 1)))
    return (e, j, q, worst)


def hexd(x):
    return float(x).hex()


def main():
    jobs = [(e, j) for e in range(0, E_LAST + 1) for j in range(2**seg_k(e))]
    with mproc.Pool(max(1, os.cpu_count() or 1)) as pool:
        res = pool.map(job, jobs, chunksize=32)
    res.sort(key=lambda r: seg_index(r[0], r[1]))
    assert len(res) == N_ALL
    worst = max(r[3] for r in res)
    print(f"fixed-point FP64 table: {len(res)} segments, emulated worst relative error {worst:.3g}",
          file=sys.stderr)
    lines = [
        "// Generated by paper_0901_0638_gb300/fit/gen_fx_tables.py -- do not edit.\n",
        "// FP64 normal quantile, exponential coordinate, segment expansions of\n",
        "// G(t) = Q(V - log(1 + t/m_c)) from the recycling ODE Q'' + Q' = Q Q'^2,\n",
        "// re-expanded about the segment end and stored for fixed-point evaluation:\n",
        "// G = a0 + t_u H, H = sum beta_k tau'^k > 0, tau' = (m_end - m) 2^K - 2^(K-52)\n",
        "// in [0, 1) (t_u = m_end - m),\n",
        "// in the half offset th = tau'/2: beta'_k = beta_k 2^k, all positive;\n",
        "// beta'_0..2 as integers B_k = beta'_k 2^-s0 (A: a0, B0, B1, B2 | e0 << 52,\n",
        "// e0 = 1083 + s0, H(0) 2^-s0 in [2^61, 2^62)),\n",
        "// beta'_3..6 as 32-bit integers C_k = beta'_k 2^-(s0 + c) (C: C3, C4, C5,\n",
        "// C6 | (32 - c) << 27).\n",
        f"// Binade e = -1 - E = 0..{E_LAST}, {2**K_MAIN} segments each; index (e + 1) 2^{K_MAIN} + j;\n",
        f"// rows 0..{2**K_MAIN - 1} (e = -1, x = 1 exactly: u = 1/2) are zero, so that z = +0 there.\n",
        f"// Emulated worst relative error over the checked points: {worst:.3g}.\n",
        "#pragma once\n#include \"qm_fx.cuh\"   // layout (K, E_LAST, N_ALL, FxTable) and evaluation\n\n",
        "namespace qm {\nnamespace fxt {\n\n",
        "__device__ const FxTable SEG_FX = {\n {\n",
    ]
    lines += ["  {0x0p+0,0ll,0ll,0ll},\n"] * 2**K_MAIN          # e = -1: a0 = 0, H = +0
    for e, j, q, _ in res:
        B = q["B"]
        b2s = (q["e0"] << 52) | B[2]
        if b2s >= 2**63:
            b2s -= 2**64
        lits = [f"{b}ll" for b in B[:2]] + [f"{b2s}ll" if b2s != -2**63 else "(-0x7fffffffffffffffll - 1)"]
        lines.append("  {" + hexd(q["a0"]) + "," + ",".join(lits) + "},\n")
    lines.append(" },\n {\n")
    lines += ["  {0u,0u,0u,0u},\n"] * 2**K_MAIN
    for e, j, q, _ in res:
        C = q["C"]
        w = C[:3] + [C[3] | (q["sh"] << 27)]
        lines.append("  {" + ",".join(f"{x:#x}u" for x in w) + "},\n")
    lines.append(" }\n};\n\n}  // namespace fxt\n}  // namespace qm\n")
    with open(OUT, "w") as f:
        f.write("".join(lines))
    print("wrote", OUT, file=sys.stderr)


if __name__ == "__main__":
    main()
