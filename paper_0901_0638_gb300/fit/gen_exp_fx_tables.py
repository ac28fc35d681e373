"""Generate csrc/qm_exp_fx_tables.h: the exponential -> normal recycling map
z = Phi^{-1}(1 - e^{-x}) on given Exp(1) samples x (Sec. 2.3, Sec. 6), with
one FP64 FMA per element.

The local expansions come from the exponential-background recycling ODE
Q'' + Q' = Q Q'^2 (rode.taylor_exp_background):

* ROWS / ROWS_IN[(E - X_EMIN) 2^K + j], 2^-26 <= x < 128, K = 6: segment j
  (the top 6 bits of the significand m) of the binade x = 2^E m, in the
  FIXED row layout (gen_fx_tables.quantise: H in the half offset, three
  64-bit Horner steps and a 32-bit inner chain, H > 0 asserted):
    below the segment [0.6875, 0.6953125) that holds ln 2:
        |z| = a0 + t_u H,  z = -|z|,  |z| = Q(y), y = -log(2(1 - e^{-x}))
        (the ODE series of Q at y_c composed with the series of y);
    from it on:
        z = a0 - t_u H,  z = Q(v), v = x - ln 2 (the ODE series at v_c).
  t_u = m_end - m is the offset back from the segment end, read from the
  significand bits as in the FIXED quantile kernel.  Each expansion is the
  centre series truncated to degree 7 and re-expanded exactly about the end.
* ROW_C, |x - ln 2| < 2^-12: z = v P(t), t = 1/32 - v, P(v) = Q(v)/v from the
  series about v = 0, re-expanded about v = 1/32, tau = 8 t, in the row form
  of qm_t_fx.h (centre_row); relative accuracy through z = 0.

Every row is checked by emulating the device's integer steps exactly against
mpmath at points of the row, and the worst relative error is printed.  Usage:
python -m paper_0901_0638_gb300.fit.gen_exp_fx_tables
"""
from __future__ import annotations

import math
import multiprocessing as mproc
import os
import struct
import sys
from fractions import Fraction as Fr

import mpmath as mp

from . import rode
from . import gen_fx_tables as FX
from . import targets as T

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(os.path.dirname(HERE), "csrc", "qm_exp_fx_tables.h")
with mp.workdps(60):
    LN2 = +mp.log(2)                  # kept at 60 digits (module import runs at mpmath's default 15)
DEG_C = 9                             # the centre row's ODE series: Q(v) to v^9, P(v) = Q(v)/v to v^8


def reexpand(c, h, sign=1):
    """Coefficients in t of sum_k c_k s^k with s = h + sign t (exact, mpmath)."""
    n = len(c)
    return [sum(c[k] * mp.binomial(k, m) * h ** (k - m) for k in range(m, n)) * sign ** m for m in range(n)]


def quantise(d, taumax, label):
    """The fixed-point row fields for P(tau) = sum d_k tau^k, tau in [0, taumax]."""
    d = list(d) + [mp.mpf(0)] * (9 - len(d))
    assert d[0] > 0, label
    for k in range(1, 9):
        if d[k] < 0:
            assert -d[k] <= mp.mpf(10) ** -18 * d[0], (label, k, float(d[k] / d[0]))
            d[k] = mp.mpf(0)
    assert sum(d[k] * mp.mpf(taumax) ** k for k in range(9)) < 2 * d[0], label
    e2 = int(mp.floor(mp.log(d[0], 2))) + 1
    s0 = e2 - 60
    D = [int(mp.nint(d[k] / mp.mpf(2) ** s0)) for k in range(5)]
    # inner chain: C_k = d_{k+5} 2^-(s0 + c) on 32-bit integers, every Horner
    # partial value (tau <= taumax) below 2^32; the shift 32 - c in the top
    # five bits of the last word
    fk = [d[k + 5] / mp.mpf(2) ** s0 for k in range(4)]

    def partial_max(v):
        return max(sum(v[i] * mp.mpf(taumax) ** (i - k) for i in range(k, 4)) for k in range(4))

    pm = partial_max(fk)
    c = max(1, int(mp.ceil(mp.log(pm, 2))) - 32) if pm > 0 else 1
    while True:
        C = [int(mp.nint(x / mp.mpf(2) ** c)) for x in fk]
        if partial_max([mp.mpf(x) for x in C]) < 2**32 - 8:
            break
        c += 1
    e0 = 1081 + s0
    assert 2**59 <= D[0] <= 2**60 and D[4] < 2**52 and 0 < e0 < 2048, label
    assert 1 <= c <= 32 and C[3] < 2**27, (label, c, C)
    return D, C[:3] + [C[3] | ((32 - c) << 27)], s0, e0


def mulhi3(a, b):
    """floor(a b / 2^64) from three 32-bit limb products, as the device forms
    it (a < 2^62, b < 2^63): the exact high half or one less."""
    a0, a1, b0, b1 = a & 0xFFFFFFFF, a >> 32, b & 0xFFFFFFFF, b >> 32
    m = a0 * b1 + a1 * b0
    assert m < 2**64
    r = a1 * b1 + (m >> 32)
    assert 0 <= ((a * b) >> 64) - r <= 1
    return r


def emulate(a0, D, w, s0, Sig, mlt):
    """The device's chain for a row: fma(mlt, P, a0) with P from Sig = tau 2^64."""
    assert 0 <= Sig < 2**63
    t32 = Sig >> 32
    a = w[3] & 0x07FFFFFF
    for ck in (w[2], w[1], w[0]):
        a = ck + ((a * t32) >> 32)
        assert a < 2**32
    acc = D[4] + ((a * t32) >> (w[3] >> 27))
    for k in (3, 2, 1, 0):
        assert acc < 2**62
        acc = D[k] + mulhi3(acc, Sig)
    assert 2**59 <= acc < 2**61
    top = acc >> 60
    pm = (acc + (64 << top)) >> (7 + top)
    P = Fr(pm) * Fr(2) ** (7 + top + s0)
    return float(Fr(mlt) * P + Fr(a0))


def sig_of(t, k):
    """floor(t 2^(64 + k)) from the double t >= 0, as the device forms it."""
    if t == 0:
        return 0
    m, e = math.frexp(t)                  # t = m 2^e, m in [0.5, 1)
    M = int(m * 2**53)                    # 53-bit significand
    sh = e - 53 + 64 + k
    return (M << sh) & (2**63 - 1) if sh >= 0 else (M >> -sh if sh > -64 else 0)


def centre_row():
    """ROW_C: z = v P(v) about v = 0, P(v) = Q(v)/v from the ODE series with
    Q(0) = 0, Q'(0) = sqrt(pi/2), re-expanded about v = 1/32 in t = 1/32 - v,
    tau = 8 t <= 3/8 (v >= -1/64), quantised in the row form of qm_t_fx.h and
    checked by emulating the device's chain at points of [-1/64, 1/32)."""
    mp.mp.dps = 40
    b = rode.taylor_exp_background(mp.mpf(0), mp.mpf(0), mp.sqrt(mp.pi / 2), DEG_C + 1)[: DEG_C + 1]
    ve = mp.mpf(1) / 32
    p = reexpand(b[1:], ve, -1)
    d = [p[i] / mp.mpf(2) ** (3 * i) for i in range(len(p))]
    D, f, s0, e0 = quantise(d, mp.mpf(3) / 8, "centre row")
    worst = 0.0
    vlo = -ve / 2
    for frac in (0.0, 0.13, 0.5, 0.87, 0.999):
        v = float(vlo + (ve - vlo) * frac)
        if v == 0.0:
            continue
        t = float(mp.mpf(float(ve)) - mp.mpf(v))         # rounded as the device rounds it
        z = emulate(0.0, D, f, s0, sig_of(t, 3), v)
        vv = mp.mpf(v)
        ref = T.q_exp(vv) if vv >= 0 else -T.q_exp(-mp.log(2 - mp.exp(-vv)))
        worst = max(worst, float(abs(mp.mpf(z) / ref - 1)))
    return 0.0, D, f, e0, worst


def q_and_slope(v):
    """Q(v) = Phi^{-1}(1 - e^{-v}/2) and Q'(v) = e^{-v} / (2 phi(Q)), the
    initial values of the exponential-background ODE series at v."""
    if v == 0:
        return mp.mpf(0), mp.sqrt(mp.pi / 2)
    q0 = T.q_exp(v)
    return q0, mp.exp(-v) / 2 / mp.npdf(q0)


K = 6                                  # 64 segments in every binade of x (the FIXED layout)
X_EMIN = -26                           # below 2^-26, u = x - x^2/2 is 1 - e^{-x} to double precision
X_EMAX = 6                             # binades 2^X_EMIN .. [64, 128) of x
NROWS = (X_EMAX - X_EMIN + 1) << K
POS_X = mp.mpf("0.6875")               # the segment [0.6875, 0.6953125) holds ln 2: z = a0 - t_u H from it on
V_NEAR = mp.mpf(2) ** -12              # |v| < V_NEAR: the centre row (z = v P)


def seg_bounds(E, j):
    lo = mp.mpf(2) ** E * (1 + mp.mpf(j) / 2**K)
    return lo, lo + mp.mpf(2) ** (E - K)


def centre_series(E, j):
    """z (signed) about the centre of segment j of the binade [2^E, 2^(E+1)),
    as a series in t = m - m_c (x = 2^E m), degree FX.DEG + 1, and the side:
    'pos' from the segment that holds ln 2 on (z = Q(v), v = x - ln 2, from
    the exponential-background ODE series at v_c), 'neg' below it
    (z = -Q(y), y = -log(2(1 - e^{-x})): the ODE series of Q at y_c composed
    with the series of y(x_c + s) - y_c)."""
    mp.mp.dps = 50
    n = FX.DEG + 2
    mlo = 1 + mp.mpf(j) / 2**K
    mc = mlo + mp.mpf(1) / 2**(K + 1)
    xc = mp.mpf(2) ** E * mc
    scale = [mp.mpf(2) ** (E * k) for k in range(n + 1)]           # s = x - x_c = 2^E t
    if mp.mpf(2) ** E * mlo >= POS_X:
        vc = xc - LN2
        q0, q1 = q_and_slope(vc)
        b = rode.taylor_exp_background(vc, q0, q1, n)
        return "pos", [b[k] * scale[k] for k in range(n + 1)]
    ec = mp.exp(-xc)
    A0 = -mp.expm1(-xc)                                            # 1 - e^{-x_c}
    w = [mp.mpf(0)] + [-ec * mp.mpf(-1) ** k / mp.factorial(k) / A0 for k in range(1, n + 1)]
    L = [mp.mpf(0)] + [mp.mpf(-1) ** (k + 1) / k for k in range(1, n + 1)]      # log(1 + w)
    dy = [-c for c in rode.compose(L, w, n)]                       # y(x_c + s) - y_c
    yc = -mp.log(2 * A0)
    q0, q1 = q_and_slope(yc)
    b = rode.taylor_exp_background(yc, q0, q1, n)
    a = rode.compose(b, dy, n)
    return "neg", [-a[k] * scale[k] for k in range(n + 1)]


def fx_h(q, Tu):
    """H of a FIXED-layout row at the integer offset Tu, as the kernel forms
    it (gen_fx_tables: the chains, the rounding shift, the bit assembly)."""
    Tp = Tu - 1
    Tau = Tp << (11 + K)
    acc = q["B"][FX.NI - 1] + FX.inner(q, Tp >> 15)
    assert acc < 2**62
    acc = q["B"][1] + FX.mulhi_limbs(acc, Tau)
    assert acc < 2**62
    acc = q["B"][0] + FX.mulhi_limbs(acc, Tau)
    assert 2**61 <= acc < 2**63
    top = acc >> 62
    mant = (acc + (256 << top)) >> (9 + top)
    return Fr(mant) * Fr(2) ** (9 + top + q["s0"])


def truth(x):
    x = mp.mpf(x)
    v = x - LN2
    if v >= 0:
        return T.q_exp(v)
    return -T.q_exp(-mp.log(2 * (-mp.expm1(-x))))


def binade_row(ij):
    """One device row: |z| = a0 + t_u H (neg side, z = -|z|) or z = a0 - t_u H
    (pos side) in the offset t_u = m_end - m back from the segment end, H with
    positive coefficients (asserted by gen_fx_tables.quantise), checked by
    emulating the kernel's arithmetic against mpmath."""
    E, j = ij
    mp.mp.dps = 50
    side, a = centre_series(E, j)
    # the centre expansion truncated to degree FX.DEG, then re-expanded exactly
    # about the segment end (the same polynomial, so the same truncation error)
    g = reexpand(a[:FX.DEG + 1], mp.mpf(1) / 2**(K + 1), -1)       # z(m_end - t_u)
    if side == "neg":
        g = [-c for c in g]                                        # |z| = a0 + t_u H
    else:
        g = [g[0]] + [-c for c in g[1:]]                           # z = a0 - t_u H
    q = FX.quantise(E, j, K, g)
    full = 2**(52 - K)
    lo, hi = seg_bounds(E, j)
    pts = [1, 2, 3, full // 3, full // 2, full - 1, full]
    if lo <= LN2 < hi:                        # both sides of |v| = V_NEAR, where this row takes over
        for vv in (V_NEAR, -V_NEAR, 2 * V_NEAR, -2 * V_NEAR, mp.mpf(2) ** -8, -mp.mpf(2) ** -8):
            pts.append(int((hi - (LN2 + vv)) / mp.mpf(2) ** (E - 52)))
    worst = 0.0
    for Tu in pts:
        x = float((hi - mp.mpf(Tu) * mp.mpf(2) ** (E - 52)))
        if x < 2.0**-26:
            continue
        if lo <= LN2 < hi and abs(mp.mpf(x) - LN2) < V_NEAR:
            continue
        tu = Fr(Tu, 2**52)
        if side == "neg":
            z = -float(tu * fx_h(q, Tu) + Fr(q["a0"]))
        else:
            z = float(Fr(q["a0"]) - tu * fx_h(q, Tu))
        ref = truth(x)
        worst = max(worst, float(abs(mp.mpf(z) / ref - 1)))
    return E, j, side, q, worst


def row_literal(a0, D, f, e0):
    """The centre row as a ttbl::SegTX initialiser."""
    d4e = D[4] | (e0 << 52)
    return ("  {" + float(a0).hex() + "," + ",".join(f"{x}ull" for x in D[:4]) + f",{d4e}ull,{{" +
            ",".join(f"{x:#x}u" for x in f) + "}},\n")


def i64(v):
    """A uint64 field as a C long long literal."""
    if v >= 2**63:
        v -= 2**64
    return f"{v}ll" if v != -2**63 else "(-0x7fffffffffffffffll - 1)"


def main():
    cells = [(E, j) for E in range(X_EMIN, X_EMAX + 1) for j in range(1 << K)]
    with mproc.Pool(max(1, os.cpu_count() or 2)) as pool:
        rows = pool.map(binade_row, cells, chunksize=8)
        centre = centre_row()
    assert len(rows) == NROWS
    near_lo, near_hi = float(LN2 - V_NEAR), float(LN2 + V_NEAR)   # ROW_C serves [near_lo, near_hi)
    clo, chi = seg_bounds(-1, int((LN2 * 2 - 1) * 2**K))
    assert clo == POS_X and clo < near_lo and near_hi < chi       # the centre row inside the ln 2 segment
    bits = lambda x: struct.unpack("<Q", struct.pack("<d", x))[0]
    wn = max(r[4] for r in rows if r[2] == "neg")
    wp = max(r[4] for r in rows if r[2] == "pos")
    wc = centre[4]                          # over v in [-1/64, 1/32), wider than it serves
    print(f"exp -> normal fixed-point rows: {NROWS} binade rows (worst below ln 2 {wn:.3g}, above {wp:.3g}), "
          f"centre row (worst {wc:.3g})", file=sys.stderr)
    L = [
        "// Generated by paper_0901_0638_gb300/fit/gen_exp_fx_tables.py -- do not edit.\n",
        "// Exponential -> normal recycling map z = Phi^{-1}(1 - e^{-x}): segment j (top 6 bits\n",
        "// of the significand) of the binade [2^E, 2^(E+1)) of x at row (E - X_EMIN) 2^X_K + j,\n",
        "// in the FIXED row layout of qm_fx.cuh (ROWS: a0, B0, B1, B2 | e0 << 52; ROWS_IN: the\n",
        "// 32-bit inner chain C3..C6 | (32 - c) << 27), H > 0 in the offset t_u back from the\n",
        "// segment end: below the segment [0.6875, 0.6953125) that holds ln 2, |z| = a0 + t_u H,\n",
        "// z < 0; from it on z = a0 - t_u H.  ROW_C (the row form of qm_t_fx.h) serves\n",
        "// |x - ln 2| < 2^-12: z = v P(tau), v = x - ln 2, tau = 8 (1/32 - v).\n",
        f"// Emulated worst relative error: below ln 2 {wn:.3g}, above {wp:.3g}, centre {wc:.3g}.\n",
        "#pragma once\n#include \"qm_fx.cuh\"\n#include \"qm_t_fx.h\"\n\nnamespace qm {\nnamespace efx {\n\n",
        f"constexpr int X_K = {K};\nconstexpr int X_EMIN = {X_EMIN};\nconstexpr int X_EMAX = {X_EMAX};\n",
        f"constexpr int NROWS = {NROWS};\n",
        f"constexpr unsigned long long POS_BITS = {bits(float(POS_X)):#x}ull;    // 0.6875: z = a0 - t_u H from here\n",
        f"constexpr unsigned long long NEAR_LO_BITS = {bits(near_lo):#x}ull;   // ln 2 - 2^-12\n",
        f"constexpr unsigned long long NEAR_HI_BITS = {bits(near_hi):#x}ull;   // ln 2 + 2^-12\n\n",
        "__device__ const fxt::SegA ROWS[NROWS] = {\n",
    ]
    for _, _, _, q, _ in rows:
        B = q["B"]
        L.append("  {" + float(q["a0"]).hex() + "," + ",".join(i64(b) for b in B[:2]) + "," +
                 i64((q["e0"] << 52) | B[2]) + "},\n")
    L.append("};\n\n__device__ const fxt::SegC ROWS_IN[NROWS] = {\n")
    for _, _, _, q, _ in rows:
        C = q["C"]
        L.append("  {" + ",".join(f"{x:#x}u" for x in C[:3] + [C[3] | (q["sh"] << 27)]) + "},\n")
    a0, D, f, e0, _ = centre
    L.append("};\n\n__device__ const ttbl::SegTX ROW_C = \n" + row_literal(a0, D, f, e0).rstrip(",\n") + ";\n")
    L.append("\n}  // namespace efx\n}  // namespace qm\n")
    with open(OUT, "w") as fh:
        fh.write("".join(L))
    print("wrote", OUT, file=sys.stderr)


if __name__ == "__main__":
    main()
