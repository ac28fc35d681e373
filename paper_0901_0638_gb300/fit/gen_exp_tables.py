"""Generate csrc/qm_exp_tables.h: the exponential -> normal recycling map
z = Q_E(x) = Phi^{-1}(1 - e^{-x}) on given Exp(1) samples x (Sec. 2.3, Sec. 6).

Three regions, each a set of local expansions of the exponential-background
recycling ODE solution Q(v) = Phi^{-1}(1 - e^{-v}/2), Q'' + Q' = Q Q'^2
(rode.taylor_exp_background), composed with the coordinate change of the
region:

* x >= ln 2 (V table): z = Q(v), v = x - ln 2.  Segments of width 1/32 on
  v in [0, 1) (segment 0 expanded at v = 0, where Q(0) = 0) and 1/8 on
  [1, 64); local variable s = v - v_c.
* ln 2 - 1/64 < x < ln 2 (Y series): z = -H(y), y = ln 2 - x,
  H(y) = Q(g(y)), g(y) = -log(2 - e^y) (so that 2(1 - e^{-x}) = e^{-g}),
  one expansion at y = 0 (H(0) = 0).
* 2^-26 <= x <= ln 2 - 1/64 (X table): z = -F(r), x = 2^E m, segment j =
  top 5 bits of m, r = m c_j - 1, F(r) = Q(g_x(x)), g_x(x) = -log(2(1 - e^{-x}));
  same entry layout and evaluation as the FP64 normal table.
Below 2^-26, u = x - x^2/2 is 1 - e^{-x} to double precision and the normal
table is used on it directly.  Usage:
python -m paper_0901_0638_gb300.fit.gen_exp_tables
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
OUT = os.path.join(os.path.dirname(HERE), "csrc", "qm_exp_tables.h")

V_FINE, V_COARSE, V_SPLIT, V_MAX = 32, 8, 1, 64
DEG_V = 9
Y_MAX_INV = 64
DEG_Y = 9
X_K, X_EMIN, DEG_X = 5, -26, 7


def q_and_slope(v):
    if v == 0:
        return mp.mpf(0), mp.sqrt(mp.pi / 2)
    q0 = T.q_exp(v)
    return q0, mp.exp(-v) / 2 / mp.npdf(q0)


def v_seg(j):
    mp.mp.dps = 40
    if j < V_FINE * V_SPLIT:
        vc = mp.mpf(0) if j == 0 else (mp.mpf(j) + mp.mpf("0.5")) / V_FINE
        half = mp.mpf(1) / (2 * V_FINE)
        lo = mp.mpf(j) / V_FINE
    else:
        k = j - V_FINE * V_SPLIT
        vc = V_SPLIT + (mp.mpf(k) + mp.mpf("0.5")) / V_COARSE
        half = mp.mpf(1) / (2 * V_COARSE)
        lo = vc - half
    q0, q1 = q_and_slope(vc)
    b = rode.taylor_exp_background(vc, q0, q1, DEG_V + 1)
    worst = mp.mpf(0)
    for v in (lo + half / 4, lo + 2 * half - mp.mpf(2) ** -30):
        ref = T.q_exp(v)
        s = v - vc
        worst = max(worst, abs(sum(b[n] * s**n for n in range(DEG_V + 1)) / ref - 1))
    return j, b[: DEG_V + 1], float(worst)


def y_series():
    mp.mp.dps = 50
    b = rode.taylor_exp_background(0, 0, mp.sqrt(mp.pi / 2), DEG_Y + 2)
    g = mp.taylor(lambda y: -mp.log(2 - mp.exp(y)), 0, DEG_Y + 2)
    g[0] = mp.mpf(0)
    h = rode.compose(b, g, DEG_Y + 2)
    worst = mp.mpf(0)
    for y in (mp.mpf(1) / (4 * Y_MAX_INV), mp.mpf(1) / Y_MAX_INV):
        ref = T.q_exp(-mp.log(2 - mp.exp(y)))
        worst = max(worst, abs(sum(h[n] * y**n for n in range(DEG_Y + 1)) / ref - 1))
    return h[: DEG_Y + 1], float(worst)


def x_seg(args):
    E, j = args
    mp.mp.dps = 50
    k = X_K
    if j == 2**k - 1:
        c = 0.5
    else:
        lo = 1.0 + j / 2.0**k
        hi = 1.0 + (j + 1) / 2.0**k
        c = float(np.float32(2.0 / (lo + hi)))
    cm = mp.mpf(c)
    gx = lambda x: -mp.log(2 * (-mp.expm1(-x)))
    xc = mp.mpf(2) ** E / cm
    V = gx(xc)
    q0, q1 = q_and_slope(V) if V > 0 else (None, None)
    if q0 is None:
        # segment entirely at or above ln 2 (not used by the kernel)
        return E, j, c, [mp.mpf(0)] * (DEG_X + 1), 0.0
    b = rode.taylor_exp_background(V, q0, q1, DEG_X + 2)
    s = mp.taylor(lambda r: gx(mp.mpf(2) ** E * (1 + r) / cm) - V, 0, DEG_X + 2)
    s[0] = mp.mpf(0)
    a = rode.compose(b, s, DEG_X + 2)
    worst = mp.mpf(0)
    mlo = 1 + mp.mpf(j) / 2**k
    mhi = 1 + mp.mpf(j + 1) / 2**k
    ln2 = mp.log(2)
    for m in (mlo, (mlo + mhi) / 2, mhi - mp.mpf(2) ** -30):
        x = m * mp.mpf(2) ** E
        if x > ln2 - mp.mpf(1) / Y_MAX_INV:
            continue
        r = m * cm - 1
        ref = T.q_exp(gx(x))
        worst = max(worst, abs(sum(a[n] * r**n for n in range(DEG_X + 1)) / ref - 1))
    return E, j, c, a[: DEG_X + 1], float(worst)


def hexd(x):
    return float(x).hex()


def hexf(x):
    return float(np.float32(float(x))).hex() + "f"


def main():
    nv = V_FINE * V_SPLIT + V_COARSE * (V_MAX - V_SPLIT)
    xjobs = [(E, j) for E in range(-1, X_EMIN - 1, -1) for j in range(2**X_K)]
    with mproc.Pool(max(1, os.cpu_count() or 2)) as pool:
        vs = pool.map(v_seg, range(nv), chunksize=8)
        xs = pool.map(x_seg, xjobs, chunksize=8)
    ys, yw = y_series()
    print(f"V table: {nv} segments, truncation <= {max(w for _, _, w in vs):.3g}", file=sys.stderr)
    print(f"Y series: truncation <= {yw:.3g}", file=sys.stderr)
    print(f"X table: {len(xs)} segments, truncation <= {max(x[4] for x in xs):.3g}", file=sys.stderr)
    L = [
        "// Generated by paper_0901_0638_gb300/fit/gen_exp_tables.py -- do not edit.\n",
        "// Exponential -> normal recycling map z = Phi^{-1}(1 - e^{-x}): local\n",
        "// expansions of the exponential-background recycling ODE (see the generator).\n",
        "#pragma once\n#include \"qm_tables.h\"\n#include \"qm_t_tables.h\"\n\nnamespace qm {\nnamespace etbl {\n\n",
        f"constexpr int V_FINE = {V_FINE};\nconstexpr int V_COARSE = {V_COARSE};\n",
        f"constexpr int V_SPLIT = {V_SPLIT};\nconstexpr int V_MAX = {V_MAX};\nconstexpr int NV = {nv};\n",
        f"constexpr int Y_MAX_INV = {Y_MAX_INV};\nconstexpr int DEG_Y = {DEG_Y};\n",
        f"constexpr int X_K = {X_K};\nconstexpr int X_EMIN = {X_EMIN};\n\n",
        f"__device__ const ttbl::SegT SEG_V[NV] = {{\n",
    ]
    for j, b, _ in vs:
        L.append("  {{" + ",".join(hexd(x) for x in b[:5]) + "},{" + ",".join(hexf(x) for x in b[5:10]) +
                 "},0.0f},\n")
    L.append("};\n\n__device__ const double Y_SERIES[DEG_Y + 1] = {" + ",".join(hexd(x) for x in ys) + "};\n\n")
    L.append(f"__device__ const tbl::SegF64 SEG_X[{len(xs)}] = {{\n")
    for E, j, c, a, _ in xs:
        L.append("  {{" + ",".join(hexd(x) for x in a[:4]) + "}," + hexd(c) + ",{" +
                 ",".join(hexf(x) for x in a[4:8]) + "},{0.0f,0.0f}},\n")
    L.append("};\n\n}  // namespace etbl\n}  // namespace qm\n")
    with open(OUT, "w") as f:
        f.write("".join(L))
    print("wrote", OUT, file=sys.stderr)


if __name__ == "__main__":
    main()
