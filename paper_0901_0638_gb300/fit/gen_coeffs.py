"""Generate csrc/qm_coeffs.h: the rational approximations of the kernels.

Every table is the builder's own minimax fit (``rational.remez``) of a function
the paper defines, in the coordinate the paper chooses:

* exponential coordinate v = -log(2 min(u, 1-u)) (Sec. 6; Sec. 7.2):
    - F64_EXP  : Q(v)/v on [0, 42], degree (13,13)  -- the branch-free FP64
                 form, same domain and degree as the paper's Sec. 7.2 model;
    - F64_DEEP : Q(v)/v on [42, 745], degree (11,11) -- extends the FP64 form
                 down to the smallest subnormal (beyond the paper's domain);
    - F32_PAPER: Q(v)/v on [0, 25], degree (5,6)     -- the paper's Sec. 6.1
                 single-precision form;
    - F32_SQRT : (Q(v)/v)^2 on [0, 25], degree (6,6) -- the same change of
                 variables, evaluated as z = v sqrt(R(v)) so that FP32 Horner
                 rounding enters the result at half weight;
    - F32_TAIL : (Q(v)/v)^2 on [25, 104], degree (3,3) -- single-precision
                 inputs below e^-25/2 down to the smallest subnormal;
    - F32_DEEP : (Q(v)/v)^2 on [104, 745], degree (3,3) -- the FP32 first
                 guess of the mixed-precision form for double inputs below the
                 single-precision range.
* scaled Student-t_2 coordinate v = |u - 1/2| / sqrt(u - u^2) (Sec. 7.3):
    - F64_T2   : Psi(v)/v on [0, 15.5], degree (14,15).

The minimax solution is unique, so where the paper prints a fit of the same
function, degree and interval, these coefficients agree with its digits to
the accuracy of the fit.  Usage:  python -m paper_0901_0638_gb300.fit.gen_coeffs
"""
from __future__ import annotations

import os
import sys

import mpmath as mp
import numpy as np

from . import rational as R
from . import targets as T

HERE = os.path.dirname(os.path.abspath(__file__))
OUT = os.path.join(os.path.dirname(HERE), "csrc", "qm_coeffs.h")


def q_over_v(v):
    return T.q_exp(v) / v if v != 0 else mp.sqrt(mp.pi / 2)


def q_over_v_sq(v):
    return (T.q_exp(v) / v) ** 2 if v != 0 else mp.pi / 2


def psi_over_v(v):
    return T.psi_t2(v) / v if v != 0 else mp.sqrt(mp.pi / 2)


def best_scale_f32(ratio):
    """A float s in [1, 2) such that s and s*ratio are both (nearly exactly)
    single-precision numbers: the leading coefficients p0 = s*ratio, q0 = s of
    a float rational then carry the exact value of P(0)/Q(0)."""
    s = (np.arange(2**23, dtype=np.float64) + 2**23) / 2**23
    prod = s * float(ratio)
    err = np.abs(prod.astype(np.float32).astype(np.float64) - prod) / prod
    i = int(np.argmin(err))
    return mp.mpf(float(s[i]))


def fit(fun, a, b, n, m):
    p, q, e, _ = R.remez(fun, a, b, n, m, ngrid=1500)
    P, Q = R.to_monomial(p, q, a, b)
    return P, Q, e


def check(fun, P, Q, a, b, cast):
    worst = mp.mpf(0)
    Pc = [mp.mpf(cast(c)) for c in P]
    Qc = [mp.mpf(cast(c)) for c in Q]
    for x in np.linspace(a, b, 1201):
        xm = mp.mpf(float(x))
        ref = fun(xm)
        worst = max(worst, abs(R.horner(Pc, xm) / R.horner(Qc, xm) / ref - 1))
    return worst


def fmt64(c):
    return repr(float(c))


def fmt32(c):
    f = np.float32(float(c))
    return np.format_float_scientific(f, unique=True, trim="-") + "f"


def table(name, coeffs, ctype, fmt):
    body = ",\n    ".join(fmt(c) for c in coeffs)
    return f"QM_COEF {ctype} {name}[{len(coeffs)}] = {{\n    {body}}};\n"


def main():
    mp.mp.dps = 40
    specs = [
        # name, fun, a, b, n, m, precision, leading ratio for f32 scaling
        ("F64_EXP", q_over_v, 0, 42, 13, 13, 64),
        ("F64_DEEP", q_over_v, 42, 745, 11, 11, 64),
        ("F64_T2", psi_over_v, 0, 15.5, 14, 15, 64),
        ("F32_PAPER", q_over_v, 0, 25, 5, 6, 32),
        ("F32_SQRT", q_over_v_sq, 0, 25, 6, 6, 32),
        ("F32_TAIL", q_over_v_sq, 25, 104, 3, 3, 32),
        ("F32_DEEP", q_over_v_sq, 104, 745, 3, 3, 32),
    ]
    out = [
        "// Generated by paper_0901_0638_gb300/fit/gen_coeffs.py -- do not edit.\n",
        "// Minimax rationals P(v)/Q(v) (monomial coefficients, constant term\n",
        "// first) of the normal quantile in the paper's transformed coordinates;\n",
        "// the generator's docstring gives each function, interval and degree.\n",
        "#pragma once\n\n#ifndef QM_COEF\n#define QM_COEF static __constant__ const\n#endif\n\n",
        "namespace qm {\nnamespace coef {\n\n",
    ]
    for name, fun, a, b, n, m, prec in specs:
        P, Q, e = fit(fun, a, b, n, m)
        if prec == 32:
            s = best_scale_f32(P[0] / Q[0])
            P = [c * s for c in P]
            Q = [c * s for c in Q]
            cast = lambda c: float(np.float32(float(c)))
            ctype, fm = "float", fmt32
        else:
            cast = lambda c: float(c)
            ctype, fm = "double", fmt64
        worst = check(fun, P, Q, a, b, cast)
        print(f"{name}: [{a},{b}] ({n},{m}) minimax {float(e):.3g}, "
              f"with rounded coefficients {float(worst):.3g}", file=sys.stderr)
        out.append(f"// {name}: [{a}, {b}], degree ({n},{m}); minimax relative error "
                   f"{float(e):.3g}, {float(worst):.3g} with {ctype} coefficients.\n")
        out.append(f"static constexpr {ctype} {name}_LO = {a};\n")
        out.append(f"static constexpr {ctype} {name}_HI = {b};\n")
        out.append(table(name + "_P", P, ctype, fm))
        out.append(table(name + "_Q", Q, ctype, fm))
        out.append("\n")
    out.append("}  // namespace coef\n}  // namespace qm\n")
    with open(OUT, "w") as f:
        f.write("".join(out))
    print("wrote", OUT, file=sys.stderr)


if __name__ == "__main__":
    main()
