"""Generate csrc/qm_filter_coeffs.h: the normal quantile through the other
filtering distributions of Sec. 4.4, and the near-tail t_2 piece of the
multi-branch hybrid (Sec. 7.4).

Almost-normal / almost-chi-squared coordinates (Sec. 4.4).  With
d = min(u, 1-u) and r = |2u - 1| = 1 - 2d, the almost-chi-squared variate
(the square of the almost-normal one) is

    a = Q_AN(u)^2 = -(pi/2) log(4 d (1 - d)) = -(pi/2) log(1 - r^2),

and w = sqrt(a) = |Q_AN(u)|.  The normal quantile is recycled from them:

* centre, a <= A0:  |Phi^{-1}(u)| = r P(a).  Phi^{-1}(1/2 + r/2)/r is an
  analytic function of r^2 = 1 - e^{-2a/pi}, hence of a, with P(0) =
  sqrt(pi/2); the factor r carries the sign-free magnitude exactly, so the
  rounding of a near the centre enters only through P'/P.
* tail, a > A0:     |Phi^{-1}(u)| = T_k(w) on pieces k of the w axis.

P and T_k are polynomials (no divide) in the centred variable a - a_c or
w - w_c, minimax in relative error (rational.remez with denominator degree
0).  FP64: degree 20 on every piece (the kernel evaluates all pieces with one
Horner loop over a per-lane coefficient row); FP32: degree 9.

Near-tail t_2 piece (Sec. 7.4): Psi(v)/v on v in [15.5, 1000] (v the scaled
t_2 coordinate), degree (14,15) -- the same form as the Sec. 7.3 centre
rational, so that the two share one evaluation with per-lane coefficients.

Usage: python -m paper_0901_0638_gb300.fit.gen_filter_coeffs
"""
from __future__ import annotations

import os
import sys

import mpmath as mp
import numpy as np

from . import rational as R
from . import targets as T

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(os.path.dirname(HERE), "csrc", "qm_filter_coeffs.h")

A0 = 8
F64_DEG = 20
F64_TAIL = [(mp.sqrt(A0), 5.2), (5.2, 9.2), (9.2, 16.0), (16.0, 34.25)]   # d down to 2^-1074
F32_DEG = 9
F32_TAIL = [(mp.sqrt(A0), 5.2), (5.2, 12.75)]                            # d down to 2^-149
T2N_LO, T2N_HI, T2N_N, T2N_M = 15.5, 1000, 14, 15


def d_and_r(a):
    """d in (0, 1/2] and r = 1 - 2d with -(pi/2) log(4 d (1-d)) = a."""
    a = mp.mpf(a)
    e = mp.exp(-2 * a / mp.pi)
    r = mp.sqrt(-mp.expm1(-2 * a / mp.pi))
    return e / (2 * (1 + r)), r


def centre_target(a):
    a = mp.mpf(a)
    if a == 0:
        return mp.sqrt(mp.pi / 2)
    d, r = d_and_r(a)
    z = mp.sqrt(2) * mp.erfinv(r) if r < mp.mpf("0.9") else T.upper_probit(d)
    return z / r


def tail_target(w):
    d, _ = d_and_r(mp.mpf(w) ** 2)
    return T.upper_probit(d)


def t2_near_target(v):
    return T.psi_t2(v) / v


def poly_fit(fun, lo, hi, deg):
    """Minimax polynomial in relative error; monomial coefficients in the
    centred variable x - c, c = (lo + hi)/2."""
    p, q, err, _ = R.remez(fun, lo, hi, deg, 0, ngrid=1500, iters=40)
    assert len(q) == 1
    c = (mp.mpf(lo) + mp.mpf(hi)) / 2
    mono = R.cheb_to_monomial(p, mp.mpf(lo) - c, mp.mpf(hi) - c)
    return c, mono, err


def check_rounded(fun, lo, hi, c, coef, dtype, n=4001):
    """Max relative error of the rounded coefficients, Horner evaluated in the
    kernel's precision (FMA emulated by one rounding per step), against the
    target in mpmath."""
    cr = [dtype(float(x)) for x in coef]
    worst = 0.0
    for k in range(n):
        x = mp.mpf(lo) + (mp.mpf(hi) - mp.mpf(lo)) * k / (n - 1)
        s = dtype(float(x - c))
        acc = cr[-1]
        for ck in reversed(cr[:-1]):
            acc = dtype(float(mp.mpf(float(acc)) * mp.mpf(float(s)) + mp.mpf(float(ck))))
        y = mp.mpf(float(acc))
        ref = fun(x)
        worst = max(worst, float(abs(y / ref - 1)))
    return worst


def fmt(v, f32=False):
    if f32:
        return repr(float(np.float32(float(v)))) + "f"
    return repr(float(v))


def main():
    mp.mp.dps = 40
    out = []
    out.append("// Generated by paper_0901_0638_gb300/fit/gen_filter_coeffs.py -- do not edit.")
    out.append("// Normal quantile through the almost-normal / almost-chi-squared filtering")
    out.append("// coordinates and the near-tail t_2 piece; the generator's docstring gives")
    out.append("// each function, interval and degree.")
    out.append("#pragma once")
    out.append("")
    out.append("namespace qm {")
    out.append("namespace filt {")
    out.append("")
    out.append(f"constexpr double AN_A0 = {A0};                     // centre: a <= AN_A0")
    out.append(f"constexpr int AN64_DEG = {F64_DEG};")
    out.append(f"constexpr int AN64_PIECES = {1 + len(F64_TAIL)};")
    out.append(f"constexpr int AN32_DEG = {F32_DEG};")
    out.append("")

    # FP64 almost-normal rows: {offset, c_0 .. c_deg}
    rows = []
    c, mono, err = poly_fit(centre_target, 0, A0, F64_DEG)
    chk = check_rounded(centre_target, 0, A0, c, mono, np.float64, n=801)
    print(f"AN64 centre [0, {A0}] deg {F64_DEG}: minimax {float(err):.3g}, rounded {chk:.3g}")
    rows.append((f"centre a in [0, {A0}]: P(a) = |z|/r", c, mono, err, chk))
    for lo, hi in F64_TAIL:
        c, mono, err = poly_fit(tail_target, lo, hi, F64_DEG)
        chk = check_rounded(tail_target, lo, hi, c, mono, np.float64, n=801)
        print(f"AN64 tail [{float(lo):.4f}, {hi}] deg {F64_DEG}: minimax {float(err):.3g}, rounded {chk:.3g}")
        rows.append((f"tail w in [{float(lo):.6g}, {hi}]: |z|", c, mono, err, chk))
    out.append("// FP64 rows {centre of the variable, c_0 .. c_20}; row 0: a, rows 1..4: w;")
    out.append("// read with a per-lane row index (global memory, L1 resident).")
    out.append(f"// tail row k covers w up to AN64_WHI[k - 1].")
    out.append("static __constant__ const double AN64_WHI[4] = {" + ", ".join(fmt(hi) for _, hi in F64_TAIL) + "};")
    out.append(f"__device__ const double AN64[{len(rows)}][{F64_DEG + 2}] = {{")
    for note, c, mono, err, chk in rows:
        out.append(f"    // {note}; minimax {float(err):.3g}, {chk:.3g} with double coefficients")
        out.append("    {" + ", ".join([fmt(c)] + [fmt(x) for x in mono]) + "},")
    out.append("};")
    out.append("")

    # FP32 almost-normal
    c, mono, err = poly_fit(centre_target, 0, A0, F32_DEG)
    chk = check_rounded(centre_target, 0, A0, c, mono, np.float32, n=801)
    print(f"AN32 centre deg {F32_DEG}: minimax {float(err):.3g}, rounded {chk:.3g}")
    out.append(f"// FP32 centre a in [0, {A0}]: P(a) = |z|/r; minimax {float(err):.3g}, "
               f"{chk:.3g} in float Horner")
    out.append(f"constexpr float AN32_C_OFF = {fmt(c, True)};")
    out.append("static __constant__ const float AN32_C[" + str(F32_DEG + 1) + "] = {" +
               ", ".join(fmt(x, True) for x in mono) + "};")
    t32 = []
    for lo, hi in F32_TAIL:
        c, mono, err = poly_fit(tail_target, lo, hi, F32_DEG)
        chk = check_rounded(tail_target, lo, hi, c, mono, np.float32, n=801)
        print(f"AN32 tail [{float(lo):.4f}, {hi}] deg {F32_DEG}: minimax {float(err):.3g}, rounded {chk:.3g}")
        t32.append((lo, hi, c, mono, err, chk))
    out.append("// FP32 tail rows {centre of w, c_0 .. c_9}; row 0 covers w up to AN32_WHI0.")
    out.append(f"constexpr float AN32_WHI0 = {fmt(t32[0][1], True)};")
    out.append(f"__device__ const float AN32_T[2][{F32_DEG + 2}] = {{")
    for lo, hi, c, mono, err, chk in t32:
        out.append(f"    // w in [{float(lo):.6g}, {hi}]; minimax {float(err):.3g}, {chk:.3g} in float Horner")
        out.append("    {" + ", ".join([fmt(c, True)] + [fmt(x, True) for x in mono]) + "},")
    out.append("};")
    out.append("")

    # near-tail t_2 rational
    p, q, err, _ = R.remez(t2_near_target, T2N_LO, T2N_HI, T2N_N, T2N_M, ngrid=1500, iters=40)
    P, Q = R.to_monomial(p, q, T2N_LO, T2N_HI)
    worst = 0.0
    Pr = [float(x) for x in P]
    Qr = [float(x) for x in Q]
    for k in range(2001):
        v = mp.mpf(T2N_LO) * (mp.mpf(T2N_HI) / T2N_LO) ** (mp.mpf(k) / 2000)
        pv = R.horner([mp.mpf(x) for x in Pr], v)
        qv = R.horner([mp.mpf(x) for x in Qr], v)
        worst = max(worst, float(abs(pv / qv / t2_near_target(v) - 1)))
    print(f"T2 near [{T2N_LO}, {T2N_HI}] ({T2N_N},{T2N_M}): minimax {float(err):.3g}, rounded {worst:.3g}")
    vhi = mp.mpf(T2N_HI)
    d1 = 1 / (2 * mp.sqrt(1 + vhi * vhi) * (mp.sqrt(1 + vhi * vhi) + vhi))
    out.append(f"// near-tail t_2: Psi(v)/v on [{T2N_LO}, {T2N_HI}], degree ({T2N_N},{T2N_M}); "
               f"minimax {float(err):.3g}, {worst:.3g} with double coefficients")
    out.append(f"constexpr double T2N_V_HI = {T2N_HI};")
    out.append(f"constexpr double T2N_D_LO = {fmt(d1)};   // d above this has v < {T2N_HI}")
    out.append(f"static __constant__ const double T2N_P[{T2N_N + 1}] = {{" + ", ".join(fmt(x) for x in P) + "};")
    out.append(f"static __constant__ const double T2N_Q[{T2N_M + 1}] = {{" + ", ".join(fmt(x) for x in Q) + "};")
    out.append("")
    out.append("}  // namespace filt")
    out.append("}  // namespace qm")
    with open(OUT, "w") as f:
        f.write("\n".join(out) + "\n")
    print("wrote", OUT)


if __name__ == "__main__":
    sys.exit(main())
