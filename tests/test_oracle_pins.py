"""Pins of the CPU FP64 oracle to things other than itself.

Each test checks the oracle against a value the paper prints (fixtures in
tests/golden/paper_values.json), a closed form, an invariant of the
definition, an independent library routine (mpmath at 50 digits, scipy,
cuRAND's header implementation of Philox), or brute-force bisection.  The
cases are chosen so that a dropped term, a flipped sign or a transposed
operand anywhere in the oracle fails at least one of them.
"""
import math
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle

mp = pytest.importorskip("mpmath")
mp.mp.dps = 50

L = oracle.lib()


def _mp_probit(u):
    """Phi^{-1}(u) at 50 digits by bracketed root finding on log(1 - Phi)."""
    u = mp.mpf(u)
    if u == mp.mpf(1) / 2:
        return mp.mpf(0)
    if u > mp.mpf(1) / 2:
        return -_mp_probit(1 - u)
    if u > mp.mpf("1e-8"):
        return -mp.sqrt(2) * mp.erfinv(1 - 2 * u)
    lu = mp.log(u)
    f = lambda w: mp.log(mp.erfc(w / mp.sqrt(2)) / 2) - lu
    lo, hi = mp.mpf(5), mp.mpf(40)
    for _ in range(190):
        mid = (lo + hi) / 2
        if f(mid) > 0:
            lo = mid
        else:
            hi = mid
    return -(lo + hi) / 2


def _rel(a, b):
    b = mp.mpf(b)
    return abs(float((mp.mpf(a) - b) / b)) if b != 0 else abs(float(a))


# ---------------------------------------------------------------- erf, erfc

def test_erf_erfc_against_mpmath():
    xs = np.concatenate([np.linspace(-6, 6, 241), np.linspace(6, 26.5, 60),
                         [1e-300, 1e-20, 1e-8, 0.7499999, 0.75, 0.7500001]])
    for x in xs:
        r = mp.erf(mp.mpf(x))
        if r != 0:
            assert _rel(L.orc_erf(x), r) < 6e-16, x
        rc = mp.erfc(mp.mpf(x))
        assert _rel(L.orc_erfc(x), rc) < 6e-16, x
    for x in np.linspace(0.75, 40, 200):
        r = mp.erfc(mp.mpf(x)) * mp.exp(mp.mpf(x) ** 2)
        assert _rel(L.orc_erfcx(x), r) < 6e-16, x


def test_erf_against_libm():
    for x in np.linspace(-5, 5, 1001):
        assert abs(L.orc_erf(x) - math.erf(x)) <= 4e-16 * max(abs(math.erf(x)), 1e-300) + 1e-300
        if x < 5:
            assert abs(L.orc_erfc(x) / math.erfc(x) - 1) < 4e-15


def test_norm_sf_and_log_form():
    for w in [0.0, 0.3, 1.0, 1.06, 2.0, 5.0, 10.0, 20.0, 37.0]:
        r = mp.ncdf(-mp.mpf(w))
        assert _rel(L.orc_norm_sf(w), r) < 8e-16, w
        assert abs(L.orc_log_norm_sf(w) - float(mp.log(r))) <= 4e-16 * max(1.0, abs(float(mp.log(r)))), w
    # deep tail where 1 - Phi underflows: log form stays exact
    for w in [38.6, 40.0, 100.0]:
        r = mp.log(mp.ncdf(-mp.mpf(w)))
        assert abs(L.orc_log_norm_sf(w) / float(r) - 1) < 4e-16


# ---------------------------------------------------------------- Phi^{-1}

U_GRID = np.concatenate([
    10.0 ** -np.linspace(0.302, 300.0, 240),      # left tail down to 1e-300
    np.linspace(0.2, 0.8, 61),                    # centre / tail boundary
    [0.25, 0.2499999999999999, 0.25000000000000006, 0.75, 0.5 + 2**-40,
     0.5 - 2**-53, 2.0**-1074, 1 - 2.0**-53, 0.975],
])


def test_probit_against_mpmath_bisection():
    z = oracle.probit(U_GRID)
    worst = 0.0
    for u, zz in zip(U_GRID, z):
        r = _mp_probit(u)
        if r == 0:
            assert zz == 0.0
            continue
        e = _rel(zz, r)
        if u < 1e-300:  # subnormal input: fewer bits in u itself
            assert e < 1e-13, u
            continue
        worst = max(worst, e)
        assert e < 8e-16, (u, zz, r)
    assert worst > 0


def test_probit_against_scipy_ndtri():
    sp = pytest.importorskip("scipy.special")
    u = np.concatenate([np.linspace(1e-6, 1 - 1e-6, 2001), 10.0 ** -np.linspace(1, 300, 300)])
    z = oracle.probit(u)
    r = sp.ndtri(u)
    assert np.all(np.abs(z - r) <= 1e-14 * np.abs(r) + 1e-300)


def test_probit_printed_values(golden):
    caps = golden["probit_right_caps"]
    tol = 0.5 * 10.0 ** -caps["printed_digits"]
    for k, printed in caps["values"]:
        # 1 - 2^-54 is not a double; by the symmetry w(1-u) = -w(u).
        w = -L.orc_probit(2.0 ** -k)
        assert abs(w - printed) <= tol, (k, w, printed)
        if k <= 53:
            assert L.orc_probit(1.0 - 2.0 ** -k) == w
    g = golden["probit_right_cap_24"]
    w24 = -L.orc_probit(2.0 ** -24)
    assert abs(w24 - g["read_as"]) <= 0.5e-4
    assert abs(w24 - g["printed"]) > 1e-2  # the printed digits are garbled
    t2 = golden["t2_filter_break"]
    v = t2["v"]
    u = 0.5 * (1.0 + v / math.sqrt(1.0 + v * v))
    assert abs(u - t2["u"]) <= 0.5e-6
    assert abs(L.orc_probit(u) - t2["psi"]) <= 0.5e-5


def test_probit_textbook_value():
    # The 97.5 % point of the standard normal.  The double nearest 0.975 is
    # 2.2e-17 below it, which moves w by that times dw/du = 1/phi(w) ~ 17.1.
    du = float(mp.mpf(0.975) - mp.mpf("0.975"))
    w = L.orc_probit(0.975)
    shift = du * math.sqrt(2 * math.pi) * math.exp(0.5 * 1.96 ** 2)
    assert abs(w - (1.959963984540054 + shift)) <= 2.3e-16


def test_probit_symmetry_bit_exact():
    k = np.array([1, 2, 3, 1000, 2**20 + 7, 2**40 + 12345, 2**52 - 1, 2**52, 2**52 + 1,
                  3 * 2**50, 2**53 - 1], dtype=np.float64)
    u = k * 2.0 ** -53
    a = oracle.probit(u)
    b = oracle.probit(1.0 - u)
    assert np.array_equal(a, -b)


def test_probit_inverts_scipy_cdf():
    sp = pytest.importorskip("scipy.special")
    u = 10.0 ** -np.linspace(0.31, 300, 500)
    w = oracle.probit(u)
    lhs = sp.log_ndtr(w)
    # |d log Phi / dw| ~ |w| in the tail: allow a few ulp of w and of log u.
    tol = 6e-16 * (np.abs(np.log(u)) + 1.0) + 4e-16 * np.abs(w) * (np.abs(w) + 1.0)
    assert np.all(np.abs(lhs - np.log(u)) <= tol)


def test_probit_edges():
    assert L.orc_probit(0.0) == -math.inf
    assert L.orc_probit(1.0) == math.inf
    assert math.isnan(L.orc_probit(math.nan))
    assert math.isnan(L.orc_probit(-1e-300))
    assert math.isnan(L.orc_probit(1.0 + 2**-52))
    z = L.orc_probit(0.5)
    assert z == 0.0 and math.copysign(1.0, z) == 1.0


def test_probit_centre_small_argument_slope():
    # Near u = 1/2: w = sqrt(2 pi) (u - 1/2) (1 + O((u-1/2)^2)).
    for e in [1e-12, 1e-9, 1e-6]:
        u = 0.5 + e
        w = L.orc_probit(u)
        slope = math.sqrt(2 * math.pi) * (u - 0.5)
        assert abs(w / slope - 1) < 2 * math.pi / 6 * e * e * 4 + 4e-16


# ---------------------------------------------------------- Student t map

def _t_from_p_nu1(p):
    return 1.0 / float(mp.tan(mp.pi * p))


def test_t_closed_forms_nu_1_2_4():
    zs = [0.05, 0.3, 0.6745, 1.0, 2.0, 3.0, 5.0, 8.5]
    for z in zs:
        zm = mp.mpf(z)
        p = mp.ncdf(-zm)                         # upper tail 1 - Phi(z)
        u = 1 - p
        # nu = 1: t = tan(pi (u - 1/2)) (Cauchy quantile)
        t1 = 1 / mp.tan(mp.pi * p)
        assert _rel(L.orc_recycle_normal_to_t(1.0, z), t1) < 2e-14, z
        # nu = 2: t = (2u - 1)/sqrt(2 u (1-u)) (Sec. 4.4, T2 quantile)
        t2 = (2 * u - 1) / mp.sqrt(2 * u * (1 - u))
        assert _rel(L.orc_recycle_normal_to_t(2.0, z), t2) < 2e-14, z
        # nu = 4: alpha = 4u(1-u); t = 2 sqrt(cos(arccos(sqrt alpha)/3)/sqrt alpha - 1)
        al = 4 * u * (1 - u)
        t4 = 2 * mp.sqrt(mp.cos(mp.acos(mp.sqrt(al)) / 3) / mp.sqrt(al) - 1)
        assert _rel(L.orc_recycle_normal_to_t(4.0, z), t4) < 2e-14, z
        assert L.orc_recycle_normal_to_t(4.0, -z) == -L.orc_recycle_normal_to_t(4.0, z)


def _rode_centre_coeffs(n, K):
    """c_0..c_K of the central series Q = sum c_k v^(2k+1) from the Sec. 3.2
    recurrence of the Gaussian-background recycling ODE, c_0 = gamma."""
    n = mp.mpf(n)
    c = [mp.sqrt(n / 2) * mp.gamma(n / 2) / mp.gamma((n + 1) / 2)]
    a = lambda l, m: (1 + 1 / n) * (2 * l + 1) * (2 * m + 1) - (2 / n) * m * (2 * m + 1)
    for i in range(K):
        s = -(2 * i + 1) * c[i]
        for l in range(i + 1):
            for m in range(i - l + 1):
                s += a(l, m) * c[i - l - m] * c[l] * c[m]
        if i >= 1:
            t = 0
            for l in range(i):
                for m in range(i - l):
                    t += (2 * m + 1) * c[i - 1 - l - m] * c[l] * c[m]
            s -= t / n
        c.append(s / ((2 * i + 3) * (2 * i + 2)))
    return c


def test_rode_recurrence_matches_printed_nu4_series(golden):
    c = _rode_centre_coeffs(4, 10)
    printed = golden["student_t_nu4"]["centre_series"]
    for k, (a, b) in enumerate(zip(c, printed)):
        assert abs(float(a) / b - 1) < 1e-15, k
    g = golden["student_t_nu4"]["gamma"]
    assert abs(float(4 / mp.mpf(3) * mp.sqrt(2 / mp.pi)) - g) < 1e-16
    assert abs(L.orc_t_gamma(4.0) / g - 1) < 4e-16
    # c1 and c2 closed forms of Sec. 3.2 for a non-integer n
    n = mp.mpf("3.7")
    c = _rode_centre_coeffs(n, 2)
    gm = c[0]
    c1 = ((n + 1) * gm**3 - n * gm) / (6 * n)
    c2 = ((7 * n**2 + 8 * n + 1) * gm**5 + (-10 * n**2 - 10 * n) * gm**3 + 3 * n**2 * gm) / (120 * n**2)
    assert abs(c[1] / c1 - 1) < 1e-40 and abs(c[2] / c2 - 1) < 1e-40


@pytest.mark.parametrize("nu", [1, 2, 3, 4, 5, 8, 10, 30])
def test_t_oracle_matches_rode_central_series(nu):
    c = _rode_centre_coeffs(nu, 40)
    for z in [1e-12, 1e-6, 0.01, 0.1, 0.25, 0.4]:
        zm = mp.mpf(z)
        s = sum(ck * zm ** (2 * k + 1) for k, ck in enumerate(c))
        assert _rel(L.orc_recycle_normal_to_t(float(nu), z), s) < 6e-15, (nu, z)


def test_t_nu4_paper_worked_example(golden):
    g = golden["student_t_nu4"]
    cs = g["centre_series"]
    zc = g["crossover"]

    def centre(z):
        y = z * z
        acc = 0.0
        for ck in reversed(cs):
            acc = acc * y + ck
        return z * acc

    def tail(z):
        w = L.orc_norm_sf(z) * g["tail_w_factor"]
        return 2.0 * w ** -0.25 * (1.0 - g["tail_c1"] * math.sqrt(w))

    worst_c, worst_all = 0.0, 0.0
    for z in np.linspace(0.01, 8.0, 800):
        t = L.orc_recycle_normal_to_t(4.0, z)
        if z < 4.0:
            worst_c = max(worst_c, abs(centre(z) / t - 1))
        approx = centre(z) if z < zc else tail(z)
        worst_all = max(worst_all, abs(approx / t - 1))
    assert worst_c < g["centre_rel_err_abs_z_lt_4"]
    assert worst_all < g["overall_rel_err"]
    # ... and the two pieces meet at the crossover with about that error
    t = L.orc_recycle_normal_to_t(4.0, zc)
    assert abs(centre(zc) / t - 1) > 0.5 * g["overall_rel_err"]
    assert abs(tail(zc) / t - 1) > 0.5 * g["overall_rel_err"]


def test_t_cornish_fisher_large_nu(golden):
    terms = golden["cornish_fisher_student"]["terms"]
    n = 30.0
    for z in [0.2, 0.5, 1.0, 1.5]:
        t = z
        for term in terms:
            poly = sum(c * z ** int(p) for p, c in term["z_coeffs"].items())
            t += poly / (term["den"] * n ** term["n_power"])
        o = L.orc_recycle_normal_to_t(n, z)
        # the first omitted term is O(z^11 / n^5)
        assert abs(t / o - 1) < 50 * max(z, 1.0) ** 10 / n ** 5, z


def test_t_against_scipy_stdtrit():
    sp = pytest.importorskip("scipy.special")
    for nu in [3.0, 5.0, 8.0, 10.0, 30.0]:
        z = np.linspace(-3.5, 3.5, 141)
        o = oracle.recycle_t(nu, z)
        r = sp.stdtrit(nu, sp.ndtr(z))
        m = np.abs(z) > 0.05
        assert np.all(np.abs(o[m] / r[m] - 1) < 1e-11), nu


def test_t_edges():
    assert L.orc_recycle_normal_to_t(3.0, 0.0) == 0.0
    assert L.orc_recycle_normal_to_t(3.0, math.inf) == math.inf
    assert math.isnan(L.orc_recycle_normal_to_t(3.0, math.nan))
    assert math.isnan(L.orc_recycle_normal_to_t(0.0, 1.0))


# ------------------------------------------------- exponential -> normal

def _exp_series(golden, v):
    acc = mp.mpf(0)
    for t in golden["exp_normal_series"]["terms"]:
        num = sum(a * mp.pi ** (j + mp.mpf(1) / 2) for j, a in enumerate(t["a"]))
        acc += t["sign"] * num / (t["den"] * mp.sqrt(2)) * mp.mpf(v) ** t["k"]
    return acc


def test_exp_to_normal_paper_series(golden):
    ln2 = math.log(2.0)
    for v in [1e-10, 1e-6, 1e-3, 0.005, 0.01, 0.02]:
        x = ln2 + v
        vv = mp.mpf(x) - mp.log(2)       # the exact offset of the double x
        s = _exp_series(golden, vv)
        bound = 4e-15 + 3.0 * float(vv) ** 10
        assert _rel(L.orc_recycle_exp_to_normal(x), s) < bound, v


def test_exp_to_normal_against_mpmath():
    xs = np.concatenate([10.0 ** -np.linspace(0, 300, 61), np.linspace(0.05, 3, 60),
                         np.linspace(3, 740, 60)])
    for x in xs:
        xm = mp.mpf(x)
        if x < math.log(2.0):           # Phi^{-1}(u), u = 1 - e^{-x} = -expm1(-x)
            r = _mp_probit(-mp.expm1(-xm))
        else:                           # Phi^{-1}(1 - e^{-x}) = -Phi^{-1}(e^{-x})
            r = -_mp_probit(mp.exp(-xm))
        if r == 0:
            continue
        assert _rel(L.orc_recycle_exp_to_normal(x), r) < 1e-15, x


def test_exp_to_normal_inverts_scipy_cdf():
    sp = pytest.importorskip("scipy.special")
    x = np.linspace(1.4, 700, 400)
    z = oracle.recycle_exp(x)
    # log(1 - Phi(z)) = -x exactly for the right tail
    assert np.all(np.abs(sp.log_ndtr(-z) + x) <= 4e-16 * x + 8e-16 * z * z)


def test_exp_to_normal_edges():
    assert L.orc_recycle_exp_to_normal(0.0) == -math.inf
    assert L.orc_recycle_exp_to_normal(math.inf) == math.inf
    assert math.isnan(L.orc_recycle_exp_to_normal(-1.0))
    assert abs(L.orc_recycle_exp_to_normal(math.log(2.0))) < 1e-16


# ---------------------------------------------------------------- Philox

def test_philox_against_curand_header(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    exe = str(tmp_path / "curand_philox_ref")
    subprocess.check_call([nvcc, "-x", "cu", "-o", exe,
                           os.path.join(root, "tests", "helpers", "curand_philox_ref.cu")])
    rng = np.random.default_rng(7)
    cases = rng.integers(0, 2**32, size=(200, 6), dtype=np.uint64)
    cases[0] = 0
    cases[1] = [2**32 - 1] * 6
    inp = "\n".join(" ".join(str(int(v)) for v in row) for row in cases) + "\n"
    out = subprocess.run([exe], input=inp, capture_output=True, text=True, check=True).stdout
    ref = np.array([[int(t) for t in line.split()] for line in out.strip().splitlines()],
                   dtype=np.uint32)
    for row, r in zip(cases, ref):
        o = oracle.philox4x32_10(row[:4].astype(np.uint32), row[4:].astype(np.uint32))
        assert np.array_equal(o, r)


def test_philox_stream_layout():
    # word i = output word (i mod 4) of the block with counter floor(i/4)
    s = oracle.philox_stream(1, 0, 12)
    for b in range(3):
        o = oracle.philox4x32_10([b, 0, 0, 0], [1, 0])
        assert np.array_equal(s[4 * b:4 * b + 4], o)
    # 64-bit counter carries into the second counter word
    i0 = (2**32 - 1) * 4
    s = oracle.philox_stream(2**33 + 5, i0, 8)
    assert np.array_equal(s[:4], oracle.philox4x32_10([2**32 - 1, 0, 0, 0], [5, 2]))
    assert np.array_equal(s[4:], oracle.philox4x32_10([0, 1, 0, 0], [5, 2]))
