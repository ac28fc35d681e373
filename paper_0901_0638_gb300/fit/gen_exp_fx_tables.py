"""Generate csrc/qm_exp_fx_tables.h: the exponential -> normal recycling map
z = Phi^{-1}(1 - e^{-x}) on given Exp(1) samples x (Sec. 2.3, Sec. 6), in the
fixed-point row form of csrc/qm_t_fx.h (one FP64 FMA per element).

The local expansions come from the exponential-background recycling ODE
Q'' + Q' = Q Q'^2 (gen_exp_tables.py), each re-expanded exactly about a
point from which |z| has non-negative coefficients (asserted for every row),
so the device runs one unsigned fixed-point chain for every lane:

* ROWS[(E - X_EMIN) 2^X_K + j], 2^-26 <= x < 128: segment j (the top X_K
  bits of the significand m) of the binade x = 2^E m, in the offset
  t_u = m_end - m back from the segment end (Tu = Tp + 1 integer,
  t_u = Tu 2^-52, tau = Tp 2^-48 in [0, 1/2)):
    below the centre segment  |z| = a0 + t_u H,   z = -|z|
                              (x_seg: Q(-log(2(1 - e^{-x}))));
    above it                  z = a0 - t_u H      (Q(v), v = x - ln 2,
                              Q' completely monotone there, so H >= 0).
* ROW_C, the centre segment [0.6875, 0.703125) that holds ln 2:
      z = v P(t),  t = 1/32 - v,  P(v) = Q(v)/v from the series about v = 0,
      re-expanded about v = 1/32, tau = 8 t (v_row(0)).
H (or P) = sum_k d_k tau^k: d_0..d_4 as integers D_k = d_k 2^-s0 (D_0 in
[2^59, 2^60]), d_5..d_8 as 32-bit integers under a per-row scale (the inner
chain), e0 = 1081 + s0 (the layout of qm_t_fx.h).  Every row is checked by
emulating the device's integer steps exactly against mpmath at points of the
row, and the worst relative error is printed.  Usage:
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
from . import targets as T
from .gen_exp_tables import DEG_V, V_COARSE, V_FINE, V_MAX, V_SPLIT, X_EMIN, X_K, q_and_slope, v_seg, x_seg

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(os.path.dirname(HERE), "csrc", "qm_exp_fx_tables.h")
NV = V_FINE * V_SPLIT + V_COARSE * (V_MAX - V_SPLIT)
NX = (-X_EMIN) << X_K
with mp.workdps(60):
    LN2 = +mp.log(2)                  # kept at 60 digits (module import runs at mpmath's default 15)


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


def v_row(j):
    mp.mp.dps = 50
    _, b, _ = v_seg(j)
    if j < V_FINE * V_SPLIT:
        w, k = mp.mpf(1) / V_FINE, 3
        vc = mp.mpf(0) if j == 0 else (mp.mpf(j) + mp.mpf("0.5")) / V_FINE
        ve = mp.mpf(j + 1) / V_FINE
    else:
        q = j - V_FINE * V_SPLIT + V_COARSE * V_SPLIT
        w, k = mp.mpf(1) / V_COARSE, 1
        vc = (mp.mpf(q) + mp.mpf("0.5")) / V_COARSE
        ve = mp.mpf(q + 1) / V_COARSE
    if j == 0:
        # z = v P(v), P(v) = sum b_{i+1} v^i about v = 0, re-expanded about
        # v = 1/32 in t = 1/32 - v
        p = reexpand(b[1:], ve, -1)
        d = [p[i] / mp.mpf(2) ** (k * i) for i in range(len(p))]
        a0 = 0.0
        taumax = mp.mpf(3) / 8                           # t <= 3/64 (v >= -1/64)
    else:
        g = reexpand(b, ve - vc, -1)                      # |z|(v_e - t) = sum g_m t^m
        a0 = float(g[0])
        H = [-g[m + 1] for m in range(len(g) - 1)]
        d = [H[i] / mp.mpf(2) ** (k * i) for i in range(len(H))]
        taumax = mp.mpf(2) ** k * w
    D, f, s0, e0 = quantise(d, taumax, ("V", j))
    # check: the device arithmetic at points of the row against mpmath
    worst = 0.0
    vlo = mp.mpf(-1) / 64 if j == 0 else ve - w
    for frac in (0.0, 0.13, 0.5, 0.87, 0.999):
        v = float(vlo + (ve - vlo) * frac)
        if j == 0 and v == 0.0:
            continue
        t = float(mp.mpf(float(ve)) - mp.mpf(v))        # exact in the device (or rounded for row 0)
        Sig = sig_of(t, k)
        mlt = v if j == 0 else -t
        z = emulate(a0, D, f, s0, Sig, mlt)
        vv = mp.mpf(v)
        ref = T.q_exp(vv) if vv >= 0 else -T.q_exp(-mp.log(2 - mp.exp(-vv)))
        worst = max(worst, float(abs(mp.mpf(z) / ref - 1)))
    return j, a0, D, f, e0, worst


def x_row(i):
    mp.mp.dps = 50
    E, j = -1 - i // (1 << X_K), i % (1 << X_K)
    _, _, c, a, _ = x_seg((E, j))
    mend = 1 + mp.mpf(j + 1) / 2**X_K
    if mp.mpf(2) ** E * (1 + mp.mpf(j) / 2**X_K) >= LN2 - mp.mpf(1) / 64:
        return i, 0.0, [2**59, 0, 0, 0, 0], [0, 0, 0, 0], 1, 0.0       # not used by the kernel
    # |z| = F(r), r = m c - 1 = (m_end c - 1) - c t_u
    cm = mp.mpf(c)
    g = reexpand(a, mend * cm - 1, -1)
    g = [g[m] * cm ** m for m in range(len(g))]           # coefficients in t_u
    a0 = float(g[0])
    Hu = [g[m + 1] for m in range(len(g) - 1)]             # H(t_u) = sum Hu_i t_u^i
    # t_u = tau / 16 + 2^-52 (tau = Tp 2^-48): H as a polynomial in tau
    h0 = mp.mpf(2) ** -52
    Ht = reexpand(Hu, h0, 1)                               # H(h0 + s), s = tau / 16
    d = [Ht[m] / mp.mpf(16) ** m for m in range(len(Ht))]
    D, f, s0, e0 = quantise(d, mp.mpf("0.5"), ("X", E, j))
    worst = 0.0
    for Tp in (0, 1, 2**23, 2**46, 2**47 - 1):
        m = mend - mp.mpf(Tp + 1) * mp.mpf(2) ** -52
        x = float(m * mp.mpf(2) ** E)
        if x >= float(LN2 - mp.mpf(1) / 64) or x < 2.0**-26:
            continue
        tu = float(mp.mpf(Tp + 1) * mp.mpf(2) ** -52)
        z = emulate(a0, D, f, s0, Tp << 16, tu)
        ref = T.q_exp(-mp.log(2 * (-mp.expm1(-mp.mpf(x)))))
        worst = max(worst, float(abs(mp.mpf(z) / ref - 1)))
    return i, a0, D, f, e0, worst


X_EMAX = 6                                      # binades 2^X_EMIN .. [64, 128) of x
NROWS = (X_EMAX - X_EMIN + 1) << X_K
C_E, C_J = -1, 12                               # the segment [0.6875, 0.703125) holds ln 2


def seg_bounds(E, j):
    lo = mp.mpf(2) ** E * (1 + mp.mpf(j) / 2**X_K)
    return lo, lo + mp.mpf(2) ** (E - X_K)


V_NEAR = mp.mpf(2) ** -12                      # |v| < V_NEAR: the centre row (z = v P)


def seg_kind(E, j):
    """'neg' below the segment that holds ln 2 (z < 0, |z| = a0 + t_u H), else
    'pos' (z = a0 - t_u H; through z = 0 in the segment of ln 2, where
    |v| >= V_NEAR keeps the cancellation below 2e-14 relative)."""
    clo, chi = seg_bounds(C_E, C_J)
    lo, hi = seg_bounds(E, j)
    return "neg" if hi <= clo else "pos"


def xp_row(E, j):
    """A row above the centre: z = a0 - t_u H(t_u) on x = 2^E m, t_u = m_end - m
    (the offset back from the segment end in the significand, t_u = (Tp + 1)
    2^-52), H with non-negative coefficients (Q' completely monotone there;
    asserted by quantise), from the ODE expansion of Q(v), v = x - ln 2, about
    the segment centre."""
    mp.mp.dps = 50
    mlo = 1 + mp.mpf(j) / 2**X_K
    mhi = mlo + mp.mpf(1) / 2**X_K
    mc = (mlo + mhi) / 2
    vc = mp.mpf(2) ** E * mc - LN2
    q0, q1 = q_and_slope(vc)
    b = rode.taylor_exp_background(vc, q0, q1, DEG_V + 1)[:DEG_V + 1]   # z in s = v - vc
    bs = [b[k] * mp.mpf(2) ** (E * k) for k in range(len(b))]          # in m - mc
    g = reexpand(bs, mhi - mc, -1)                                      # z(m_end - t_u)
    a0 = float(g[0])
    H = [-g[m + 1] for m in range(len(g) - 1)]
    Ht = reexpand(H, mp.mpf(2) ** -52, 1)                               # t_u = 2^-52 + tau / 16
    d = [Ht[m] / mp.mpf(16) ** m for m in range(len(Ht))]
    D, f, s0, e0 = quantise(d, mp.mpf("0.5"), ("XP", E, j))
    worst = 0.0
    pts = [0, 1, 2**23, 2**46, 2**47 - 1]
    if (E, j) == (C_E, C_J):                    # both sides of |v| = V_NEAR, where this row takes over
        for vv in (V_NEAR, -V_NEAR, 2 * V_NEAR, -2 * V_NEAR, mp.mpf(2) ** -8, -mp.mpf(2) ** -8):
            pts.append(int((mhi - (LN2 + vv) / mp.mpf(2) ** E) * mp.mpf(2) ** 52) - 1)
    for Tp in pts:
        m = mhi - mp.mpf(Tp + 1) * mp.mpf(2) ** -52
        x = float(m * mp.mpf(2) ** E)
        tu = float(mp.mpf(Tp + 1) * mp.mpf(2) ** -52)
        z = emulate(a0, D, f, s0, Tp << 16, -tu)
        v = mp.mpf(x) - LN2
        ref = T.q_exp(v) if v >= 0 else -T.q_exp(-mp.log(2 - mp.exp(-v)))
        worst = max(worst, float(abs(mp.mpf(z) / ref - 1)))
    return a0, D, f, e0, worst


def xn_row(E, j):
    """A row below the centre: |z| = a0 + t_u H (the X rows of x_seg)."""
    i = (-1 - E) * (1 << X_K) + j
    _, a0, D, f, e0, worst = x_row(i)
    return a0, D, f, e0, worst


def unified_row(ij):
    E, j = ij
    kind = seg_kind(E, j)
    a0, D, f, e0, worst = (xp_row if kind == "pos" else xn_row)(E, j)
    return E, j, kind, a0, D, f, e0, worst


def row_literal(a0, D, f, e0):
    d4e = D[4] | (e0 << 52)
    return ("  {" + float(a0).hex() + "," + ",".join(f"{x}ull" for x in D[:4]) + f",{d4e}ull,{{" +
            ",".join(f"{x:#x}u" for x in f) + "}},\n")


def main():
    cells = [(E, j) for E in range(X_EMIN, X_EMAX + 1) for j in range(1 << X_K)]
    with mproc.Pool(max(1, os.cpu_count() or 2)) as pool:
        rows = pool.map(unified_row, cells, chunksize=4)
        centre = v_row(0)
    clo, chi = seg_bounds(C_E, C_J)
    assert clo < LN2 - V_NEAR and LN2 + V_NEAR < chi            # the centre row inside that segment
    near_lo, near_hi = float(LN2 - V_NEAR), float(LN2 + V_NEAR)   # ROW_C serves [near_lo, near_hi)
    bits = lambda x: struct.unpack("<Q", struct.pack("<d", x))[0]
    wn = max(r[7] for r in rows if r[2] == "neg")
    wp = max(r[7] for r in rows if r[2] == "pos")
    wc = centre[5]                          # over v in [-1/64, 1/32), wider than it serves
    print(f"exp -> normal fixed-point rows: {NROWS} binade rows (worst below ln 2 {wn:.3g}, above {wp:.3g}), "
          f"centre row (worst {wc:.3g})", file=sys.stderr)
    L = [
        "// Generated by paper_0901_0638_gb300/fit/gen_exp_fx_tables.py -- do not edit.\n",
        "// Exponential -> normal recycling map z = Phi^{-1}(1 - e^{-x}) in the fixed-point\n",
        "// row form of qm_t_fx.h: ROWS[(E - X_EMIN) 2^X_K + j] for segment j of the binade\n",
        "// [2^E, 2^(E+1)) of x, in the offset t_u back from the segment end (below the\n",
        "// segment [0.6875, 0.703125) that holds ln 2, |z| = a0 + t_u H, z < 0; from it on\n",
        "// z = a0 - t_u H), and ROW_C for |x - ln 2| < 2^-12 (z = v P(tau), v = x - ln 2,\n",
        "// tau = 8 (1/32 - v)); see the generator.\n",
        f"// Emulated worst relative error: below ln 2 {wn:.3g}, above {wp:.3g}, centre {wc:.3g}.\n",
        "#pragma once\n#include \"qm_t_fx.h\"\n\nnamespace qm {\nnamespace efx {\n\n",
        f"constexpr int X_K = {X_K};\nconstexpr int X_EMIN = {X_EMIN};\nconstexpr int X_EMAX = {X_EMAX};\n",
        f"constexpr int NROWS = {NROWS};\n",
        "constexpr unsigned long long POS_BITS = 0x3FE6000000000000ull;    // 0.6875: z = a0 - t_u H from here\n",
        f"constexpr unsigned long long NEAR_LO_BITS = {bits(near_lo):#x}ull;   // ln 2 - 2^-12\n",
        f"constexpr unsigned long long NEAR_HI_BITS = {bits(near_hi):#x}ull;   // ln 2 + 2^-12\n\n",
        "__device__ const ttbl::SegTX ROWS[NROWS] = {\n",
    ]
    for _, _, _, a0, D, f, e0, _ in rows:
        L.append(row_literal(a0, D, f, e0))
    _, a0, D, f, e0, _ = centre
    L.append("};\n\n__device__ const ttbl::SegTX ROW_C = \n" + row_literal(a0, D, f, e0).rstrip(",\n") + ";\n")
    L.append("\n}  // namespace efx\n}  // namespace qm\n")
    with open(OUT, "w") as fh:
        fh.write("".join(L))
    print("wrote", OUT, file=sys.stderr)


if __name__ == "__main__":
    main()
