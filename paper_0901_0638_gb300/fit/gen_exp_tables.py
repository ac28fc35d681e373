"""Local expansions of the exponential -> normal recycling map
z = Q_E(x) = Phi^{-1}(1 - e^{-x}) on given Exp(1) samples x (Sec. 2.3, Sec. 6),
used by gen_exp_fx_tables.py (which writes the device rows).

Each is a local expansion of the exponential-background recycling ODE
solution Q(v) = Phi^{-1}(1 - e^{-v}/2), Q'' + Q' = Q Q'^2
(rode.taylor_exp_background), composed with the coordinate change of the
region:

* x >= ln 2 (v_seg): z = Q(v), v = x - ln 2.  Segments of width 1/32 on
  v in [0, 1) (segment 0 expanded at v = 0, where Q(0) = 0) and 1/8 on
  [1, 64); local variable s = v - v_c.  The device rows use segment 0 (the
  centre row); above it they take q_and_slope and the ODE series directly
  at the centres of binade segments of x (gen_exp_fx_tables.xp_row).
* 2^-26 <= x <= ln 2 - 1/64 (x_seg): z = -F(r), x = 2^E m, segment j =
  top 5 bits of m, r = m c_j - 1, F(r) = Q(g_x(x)), g_x(x) = -log(2(1 - e^{-x})).
* y_series: the expansion at x = ln 2 in y = ln 2 - x (no longer used on the
  device: segment 0 of the V expansions covers v >= -1/64 instead).
Below 2^-26, u = x - x^2/2 is 1 - e^{-x} to double precision and the normal
table is used on it directly.
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
