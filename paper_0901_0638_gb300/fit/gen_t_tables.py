"""Generate csrc/qm_t_tables.h: the normal -> Student-t recycling map tables.

Q_nu(z) = F_nu^{-1}(Phi(z)) (Sec. 3) is odd; for 0 <= z < Z1 = 8.75 it is
stored as local Taylor expansions on segments of width h = 1/32, centred at
z_c = (j + 1/2) h, except segment 0, expanded at z_c = 0 (the central series
of Sec. 3.2, odd in z).  Each expansion comes from the Gaussian-background
recycling ODE of Sec. 3.1,
    (1 + Q^2/n)(Q'' + z Q') = (1 + 1/n) Q Q'^2,
started from Q(z_c) and Q'(z_c) = phi(z_c) / f_nu(Q(z_c)) -- the recurrence of
Sec. 3.2 taken at z_c instead of 0 (rode.taylor_gauss_background_t).

For z >= Z1 the tail coordinate of Sec. 3.3 / 3.5 is used:
    w = kappa (1 - Phi(z)),  kappa = nu sqrt(pi) Gamma(nu/2) / Gamma((nu+1)/2),
    Q = sqrt(nu) w^{-1/nu} R(y),  y = w^{2/nu},
with R(0) = 1 and R'(0) = -(nu+1)/(2(nu+2)) (the paper's two-term formula)
imposed; the remaining coefficients of R are a least-squares fit on
y in [0, y(Z1)].

Per segment: a0..a4 (double) and a5..a9 (float; their terms are below 1e-6
of the result).  Usage: python -m paper_0901_0638_gb300.fit.gen_t_tables
"""
from __future__ import annotations

import multiprocessing as mproc
import os
import sys

import mpmath as mp
import numpy as np

from . import rode

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(os.path.dirname(HERE), "csrc", "qm_t_tables.h")

NU_SET = (1, 2, 3, 4, 5, 8, 10, 30)
H_INV = 32
NSEG = 280                 # Z1 = NSEG / H_INV = 8.75
DEG = 9
TAIL_DEG = 14


def t_quantile_upper(nu, p):
    """t > 0 with P(T_nu > t) = p (0 < p < 1/2), 40 digits, by bisection on
    s = log x, x = nu/(nu + t^2), of I_x(nu/2, 1/2) = 2p."""
    nu = mp.mpf(nu)
    target = mp.log(2 * p)
    f = lambda s: mp.log(mp.betainc(nu / 2, mp.mpf(1) / 2, 0, mp.exp(s), regularized=True)) - target
    lo, hi = mp.mpf(-3000), mp.mpf(0)
    # tighten the bracket with the leading tail behaviour before bisecting
    guess = (target + mp.log(nu / 2) + mp.log(mp.beta(nu / 2, mp.mpf(1) / 2))) / (nu / 2)
    for g in (guess - 5, guess + 5):
        if lo < g < hi:
            if f(g) > 0:
                hi = min(hi, g)
            else:
                lo = max(lo, g)
    for _ in range(200):
        mid = (lo + hi) / 2
        if f(mid) > 0:
            hi = mid
        else:
            lo = mid
        if hi - lo < mp.mpf(10) ** -32:
            break
    s = (lo + hi) / 2
    x = mp.exp(s)
    return mp.sqrt(nu * (1 - x) / x)


def t_map(nu, z):
    z = mp.mpf(z)
    if z == 0:
        return mp.mpf(0)
    return t_quantile_upper(nu, mp.ncdf(-z))


def t_density(nu, t):
    nu = mp.mpf(nu)
    return (mp.gamma((nu + 1) / 2) / (mp.sqrt(nu * mp.pi) * mp.gamma(nu / 2)) *
            (1 + t * t / nu) ** (-(nu + 1) / 2))


def kappa(nu):
    nu = mp.mpf(nu)
    return nu * mp.sqrt(mp.pi) * mp.gamma(nu / 2) / mp.gamma((nu + 1) / 2)


def seg(args):
    nu, j = args
    mp.mp.dps = 40
    # segment 0 is expanded at z = 0: the odd central series of Sec. 3.2
    # (Q(0) = 0, Q'(0) = gamma), which keeps relative accuracy as z -> 0
    zc = mp.mpf(0) if j == 0 else (mp.mpf(j) + mp.mpf("0.5")) / H_INV
    q0 = t_map(nu, zc)
    q1 = mp.npdf(zc) / t_density(nu, q0)
    b = rode.taylor_gauss_background_t(nu, zc, q0, q1, DEG + 1)
    worst = mp.mpf(0)
    if j % 16 == 0 or j == NSEG - 1:
        ends = ((mp.mpf(1) / (4 * H_INV), mp.mpf(1) / H_INV) if j == 0 else
                (-mp.mpf(1) / (2 * H_INV), mp.mpf(1) / (2 * H_INV)))
        for s in ends:
            ref = t_map(nu, zc + s)
            if ref != 0:
                approx = sum(b[n] * s**n for n in range(DEG + 1))
                worst = max(worst, abs(approx / ref - 1))
    return nu, j, b[: DEG + 1], float(worst)


def tail_fit(nu):
    mp.mp.dps = 40
    k = kappa(nu)
    z1 = mp.mpf(NSEG) / H_INV
    y1 = (k * mp.ncdf(-z1)) ** (mp.mpf(2) / nu)
    ys, Rs = [], []
    M = 80
    for i in range(M):
        # Chebyshev-spaced y in (0, y1], mapped back to p
        y = y1 * (1 - mp.cos(mp.pi * (i + mp.mpf(1) / 2) / M)) / 2
        w = y ** (mp.mpf(nu) / 2)
        p = w / k
        t = t_quantile_upper(nu, p)
        ys.append(y)
        Rs.append(t / (mp.sqrt(nu) * w ** (-mp.mpf(1) / nu)))
    # R(0) = 1 and R'(0) = -(nu+1)/(2(nu+2)) fixed (the Sec. 3.5 two-term
    # formula); least squares for the rest in the scaled variable y/y1, with
    # only as many terms as y1 needs for 1e-17 (none beyond y when y1 is tiny)
    r1 = -mp.mpf(nu + 1) / (2 * (nu + 2))
    deg = int(min(TAIL_DEG, max(1, mp.ceil(mp.mpf(17) / -mp.log10(y1)))))
    R = [mp.mpf(1), r1]
    if deg >= 2:
        A = mp.matrix(M, deg - 1)
        rhs = mp.matrix(M, 1)
        for i in range(M):
            for c in range(deg - 1):
                A[i, c] = (ys[i] / y1) ** (c + 2)
            rhs[i] = Rs[i] - 1 - r1 * ys[i]
        coef = mp.lu_solve(A.T * A, A.T * rhs)
        R += [coef[c] / y1 ** (c + 2) for c in range(deg - 1)]
    R += [mp.mpf(0)] * (TAIL_DEG + 1 - len(R))
    worst = max(abs(sum(R[c] * ys[i] ** c for c in range(TAIL_DEG + 1)) / Rs[i] - 1) for i in range(M))
    return nu, R, float(worst), float(y1)


def hexd(x):
    return float(x).hex()


def hexf(x):
    return float(np.float32(float(x))).hex() + "f"


def main():
    jobs = [(nu, j) for nu in NU_SET for j in range(NSEG)]
    with mproc.Pool(max(1, os.cpu_count() or 2)) as pool:
        segs = pool.map(seg, jobs, chunksize=8)
        tails = pool.map(tail_fit, NU_SET)
    worst = {}
    for nu, j, b, w in segs:
        worst[nu] = max(worst.get(nu, 0.0), w)
    for nu, R, w, y1 in tails:
        r1 = float(R[1])
        nz = sum(1 for c in R if c != 0)
        print(f"nu={nu}: segment truncation <= {worst[nu]:.3g}; tail fit {w:.3g} on y <= {y1:.3g} "
              f"with {nz} terms", file=sys.stderr)
    lines = [
        "// Generated by paper_0901_0638_gb300/fit/gen_t_tables.py -- do not edit.\n",
        "// Normal -> Student-t recycling map Q_nu(z) = F_nu^{-1}(Phi(z)) for the nu\n",
        "// in T_NU: local expansions from the Gaussian-background recycling ODE on\n",
        f"// segments of width 1/{H_INV} of 0 <= z < {NSEG / H_INV}, and the tail polynomial R(y),\n",
        "// Q = sqrt(nu) w^{-1/nu} R(w^{2/nu}), w = kappa (1 - Phi(z)).\n",
        "#pragma once\n\nnamespace qm {\nnamespace ttbl {\n\n",
        f"constexpr int NNU = {len(NU_SET)};\nconstexpr int H_INV = {H_INV};\n",
        f"constexpr int NSEG = {NSEG};\nconstexpr int TAIL_DEG = {TAIL_DEG};\n",
        "constexpr double T_NU[NNU] = {" + ",".join(f"{nu}.0" for nu in NU_SET) + "};\n",
        "__device__ const double T_NU_DEV[NNU] = {" + ",".join(f"{nu}.0" for nu in NU_SET) + "};\n\n",
        "struct alignas(64) SegT { double a[5]; float b[5]; float pad; };\n\n",
        f"__device__ const SegT SEG_T[NNU * NSEG] = {{\n",
    ]
    order = {nu: i for i, nu in enumerate(NU_SET)}
    segs.sort(key=lambda s: (order[s[0]], s[1]))
    for nu, j, b, _ in segs:
        lines.append("  {{" + ",".join(hexd(x) for x in b[:5]) + "},{" +
                     ",".join(hexf(x) for x in b[5:10]) + "},0.0f},\n")
    lines.append("};\n\n")
    lines.append("// kappa_nu, log kappa_nu, and R_nu coefficients (constant term first)\n")
    lines.append("__device__ const double T_KAPPA[NNU] = {" +
                 ",".join(hexd(kappa(nu)) for nu in NU_SET) + "};\n")
    tails.sort(key=lambda t: order[t[0]])
    lines.append(f"__device__ const double T_TAIL[NNU][TAIL_DEG + 1] = {{\n")
    for nu, R, _, _ in tails:
        lines.append("  {" + ",".join(hexd(c) for c in R) + "},\n")
    lines.append("};\n\n}  // namespace ttbl\n}  // namespace qm\n")
    with open(OUT, "w") as f:
        f.write("".join(lines))
    print("wrote", OUT, file=sys.stderr)


if __name__ == "__main__":
    main()
