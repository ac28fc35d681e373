"""The other filtering distributions of Sec. 4.4 and the near-tail t_2 piece
of Sec. 7.4, on the CPU.

* The almost-normal law as the paper defines it (density, distribution and
  closed-form quantile) is checked against itself the way the paper's
  formulas must fit together: F_AN(Q_AN(u)) = u, the density integrates to 1
  and is the derivative of F_AN, the almost-chi-squared quantile is the square
  of the almost-normal one under r = |2u - 1| (the 2-1 mapping), and F_AN is
  close to Phi.
* The generated coefficient tables (csrc/qm_filter_coeffs.h), evaluated in
  numpy in the kernels' order, are checked against the oracle's Phi^{-1}.
"""
import math
import os
import re

import mpmath as mp
import numpy as np
import pytest
from scipy import integrate, special

import oracle
from paper_0901_0638_gb300 import workloads as W


def _read_text(path):
    with open(path) as fh:
        return fh.read()


HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_0901_0638_gb300", "csrc", "qm_filter_coeffs.h")


# ------------------------------------------------------------- the paper's law

def f_an(x):
    e = math.exp(-2 * x * x / math.pi)
    return e * abs(x) / (math.pi * math.sqrt(-math.expm1(-2 * x * x / math.pi))) if x != 0 else 1 / math.sqrt(2 * math.pi)


def F_an(x):
    return 0.5 + 0.5 * math.copysign(1.0, x) * math.sqrt(-math.expm1(-2 * x * x / math.pi))


def Q_an(u):
    return math.copysign(1.0, u - 0.5) * math.sqrt(-(math.pi / 2) * math.log(4 * u * (1 - u)))


def Q_ac(u):
    return -(math.pi / 2) * math.log1p(-u * u)


def test_almost_normal_law_is_consistent():
    mp.mp.dps = 50
    for u in ("1e-12", "1e-4", "0.01", "0.2", "0.4999", "0.5001", "0.7", "0.97", "0.999999999"):
        u = mp.mpf(u)
        q = mp.sign(u - 0.5) * mp.sqrt(-(mp.pi / 2) * mp.log(4 * u * (1 - u)))        # Q_AN
        F = 0.5 + 0.5 * mp.sign(q) * mp.sqrt(1 - mp.exp(-2 * q * q / mp.pi))           # F_AN
        assert abs(F - u) < mp.mpf(10) ** -45
        r = abs(2 * u - 1)
        assert abs(-(mp.pi / 2) * mp.log(1 - r * r) - q * q) < mp.mpf(10) ** -30        # Q_AC(r) = Q_AN^2
    for u in (1e-9, 0.3, 0.5, 0.8):
        assert abs(F_an(Q_an(u)) - u) < 1e-15
    tot = integrate.quad(f_an, -np.inf, 0, epsabs=0, epsrel=1e-12, limit=200)[0] + \
        integrate.quad(f_an, 0, np.inf, epsabs=0, epsrel=1e-12, limit=200)[0]
    assert abs(tot - 1) < 1e-10
    for x in (-3.0, -0.7, 0.3, 1.1, 2.5):
        h = 1e-6
        assert abs((F_an(x + h) - F_an(x - h)) / (2 * h) - f_an(x)) < 1e-8
    xs = np.linspace(-6, 6, 2001)
    dev = max(abs(F_an(x) - special.ndtr(x)) for x in xs)
    assert dev < 5e-3          # "very close to a standard Gaussian"


# ------------------------------------------------------------- generated tables

def c_array(text, name):
    m = re.search(r"\b" + name + r"\s*(\[[^\]]*\])*\s*=\s*\{", text)
    assert m, name
    i, depth = m.end() - 1, 0
    for j in range(i, len(text)):
        depth += text[j] == "{"
        depth -= text[j] == "}"
        if depth == 0:
            break
    body = text[i:j + 1]
    return [float(x.rstrip("f")) for x in re.findall(r"[-+]?\d+\.?\d*(?:[eE][-+]?\d+)?f?", body)]


def c_scalar(text, name):
    m = re.search(r"\b" + name + r"\s*=\s*([-+0-9.eE]+)f?;", text)
    return float(m.group(1))


@pytest.fixture(scope="module")
def tables():
    text = re.sub(r"//[^\n]*", "", _read_text(HDR))
    deg64 = int(c_scalar(text, "AN64_DEG"))
    deg32 = int(c_scalar(text, "AN32_DEG"))
    return {
        "A0": c_scalar(text, "AN_A0"),
        "AN64": np.array(c_array(text, "AN64")).reshape(-1, deg64 + 2),
        "WHI64": np.array(c_array(text, "AN64_WHI")),
        "AN32_C": np.array(c_array(text, "AN32_C"), dtype=np.float32),
        "AN32_OFF": np.float32(c_scalar(text, "AN32_C_OFF")),
        "AN32_T": np.array(c_array(text, "AN32_T"), dtype=np.float32).reshape(2, deg32 + 2),
        "WHI32": np.float32(c_scalar(text, "AN32_WHI0")),
        "T2N_P": np.array(c_array(text, "T2N_P")),
        "T2N_Q": np.array(c_array(text, "T2N_Q")),
        "T2N_D_LO": c_scalar(text, "T2N_D_LO"),
    }


def an64(t, d):
    """The FP64 kernel's evaluation: one Horner loop over the lane's row."""
    t4 = (2 * d) * (2 - 2 * d)
    a = np.maximum(-(math.pi / 2) * np.log(t4), 0.0)
    centre = a <= t["A0"]
    w = np.sqrt(a)
    row = np.where(centre, 0, 1 + (w > t["WHI64"][0]) + (w > t["WHI64"][1]) + (w > t["WHI64"][2]))
    c = t["AN64"][row]
    s = np.where(centre, a, w) - c[:, 0]
    acc = c[:, -1].copy()
    for k in range(c.shape[1] - 2, 0, -1):
        acc = acc * s + c[:, k]
    return np.where(centre, 1 - 2 * d, 1.0) * acc


def an32(t, d):
    """The FP32 kernel's evaluation in float32 (the logarithm in float64,
    rounded: the device's MUFU logarithm is not emulated)."""
    d = d.astype(np.float32)
    t4 = (np.float32(2) * d) * (np.float32(2) - np.float32(2) * d)
    a = np.maximum(np.float32(-(math.pi / 2)) * np.log(t4.astype(np.float64)).astype(np.float32), np.float32(0))
    out = np.empty_like(d)
    cm = a <= np.float32(t["A0"])
    s = a[cm] - t["AN32_OFF"]
    acc = np.full(s.shape, t["AN32_C"][-1], dtype=np.float32)
    for ck in t["AN32_C"][-2::-1]:
        acc = acc * s + ck
    out[cm] = (np.float32(1) - np.float32(2) * d[cm]) * acc
    w = np.sqrt(a[~cm])
    c = t["AN32_T"][(w > t["WHI32"]).astype(int)]
    s = w - c[:, 0]
    acc = c[:, -1].copy()
    for k in range(c.shape[1] - 2, 0, -1):
        acc = acc * s + c[:, k]
    out[~cm] = acc
    return out


def d_points():
    rng = np.random.default_rng(31)
    k = rng.integers(1, 2**52, size=200000, dtype=np.int64)
    d_uni = k.astype(np.float64) * 2.0**-53
    u_mix = W.mixture_f64(2, 1 << 16).numpy()
    d_mix = np.minimum(u_mix, 1 - u_mix)
    e = np.arange(1, 1074)
    d_bin = np.concatenate([np.ldexp(0.75, -e), np.ldexp(0.5000001, -e)])
    d = np.concatenate([d_uni, d_mix, d_bin, [0.5, 0.5 - 2**-54, 0.25]])
    return d[(d > 0) & (d <= 0.5)]


def test_an64_tables_against_the_oracle(tables):
    d = d_points()
    z = an64(tables, d)
    w = -oracle.probit(d)                       # |Phi^{-1}(d)|
    nz = w != 0
    rel = np.abs(z[nz] / w[nz] - 1)
    assert rel.max() < 1.5e-15, (d[nz][np.argmax(rel)], rel.max())
    assert np.all(z[~nz] == 0)


def test_an32_tables_against_the_oracle(tables):
    d = d_points()
    d = d[d >= 2.0**-149].astype(np.float32)
    d = d[d > 0]
    z = an32(tables, d).astype(np.float64)
    w = -oracle.probit(d.astype(np.float64))
    ulp = np.spacing(np.abs(w).astype(np.float32)).astype(np.float64)
    err = np.abs(z - w) / ulp
    small = np.abs(w) < 1e-2
    assert err[~small].max() < 3.0, (d[~small][np.argmax(err[~small])], err[~small].max())
    assert np.abs(z - w)[small].max() < 2e-7


def test_t2_near_tail_rational_against_the_oracle(tables):
    v = np.geomspace(15.5, 1000, 20001)
    r = np.sqrt(1 + v * v)
    d = 1 / (2 * r * (r + v))                   # 1 - (1 + v/r)/2 without cancellation
    P = np.polynomial.polynomial.polyval(v, tables["T2N_P"])
    Q = np.polynomial.polynomial.polyval(v, tables["T2N_Q"])
    z = v * P / Q
    w = -oracle.probit(d)
    rel = np.abs(z / w - 1)
    assert rel.max() < 2e-15, (v[np.argmax(rel)], rel.max())
    # the domain constant is the d of v = 1000
    vhi = 1000.0
    assert abs(tables["T2N_D_LO"] * 2 * math.sqrt(1 + vhi * vhi) * (math.sqrt(1 + vhi * vhi) + vhi) - 1) < 1e-15
