"""CPU checks of the fixed-point segment rows that the FP64 kernels evaluate
(no GPU): the generated tables -- csrc/qm_fx_tables.h for the normal
quantile (the exponential coordinate of Sec. 6 / Sec. 7.2, expansions from
the recycling ODE of Sec. 2.3) and csrc/qm_exp_fx_tables.h for the
exponential -> normal map -- read as text, the device arithmetic emulated
exactly on Python integers (high products from three 32-bit limb
products, the 32-bit inner chain, the one-bit normalisation and the bit
assembly of the polynomial's value, the final FMA rounded once), and the
results compared with the oracle at the library's bars (4e-15 for the
normal quantile, 1e-12 for the recycled map).  The inputs cover the top
binade's segments next to u = 1/2, segment boundaries, the tail-stress
mixture's binades down to subnormal d, and mirrored u >= 1/2."""
import os
import re
import struct
from fractions import Fraction as Fr

import numpy as np
import pytest

import oracle


def _read_text(path):
    with open(path) as fh:
        return fh.read()


CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_0901_0638_gb300", "csrc")
M64 = (1 << 64) - 1
MANT = (1 << 52) - 1


def bits(x: float) -> int:
    return struct.unpack("<Q", struct.pack("<d", x))[0]


def dbl(b: int) -> float:
    return struct.unpack("<d", struct.pack("<Q", b & M64))[0]


def mulhi3(a: int, b: int) -> int:
    """The kernels' high product: a1 b1 + hi32(a0 b1 + a1 b0), a < 2^62, b < 2^63."""
    assert 0 <= a < 2**62 and 0 <= b < 2**63
    a0, a1, b0, b1 = a & 0xFFFFFFFF, a >> 32, b & 0xFFFFFFFF, b >> 32
    m = a0 * b1 + a1 * b0
    assert m < 2**64
    r = a1 * b1 + (m >> 32)
    assert 0 <= ((a * b) >> 64) - r <= 1          # exact or one unit low
    return r


def inner(w, t32: int) -> int:
    """32-bit inner chain on (C_a, C_b, C_c, C_d | sh << 27), Horner, and its
    join floor(C t32 / 2^sh)."""
    x = w[3] & 0x07FFFFFF
    for ck in (w[2], w[1], w[0]):
        x = ck + ((x * t32) >> 32)
        assert x < 2**32
    return (x * t32) >> (w[3] >> 27)


def _int(tok: str) -> int:
    tok = tok.strip()
    if tok.startswith("("):                           # (-0x7fffffffffffffffll - 1)
        return -(2**63)
    return int(tok.rstrip("ul").rstrip("l"), 0)


@pytest.fixture(scope="module")
def fx_table():
    """(A rows: a0 bits, B0, B1, B2 | e0;  C rows: four 32-bit words)."""
    text = _read_text(os.path.join(CSRC, "qm_fx_tables.h"))
    body = text[text.index("SEG_FX = {"):]
    a_part, c_part = body.split(" },\n {\n", 1)
    A = []
    for m in re.finditer(r"\{(0x[0-9a-fp.+-]+|[-0-9.e+]+),([^,{}]+),([^,{}]+),([^{}]+)\}", a_part):
        A.append((bits(float.fromhex(m.group(1))), _int(m.group(2)) & M64, _int(m.group(3)) & M64,
                  _int(m.group(4)) & M64))
    C = [tuple(int(x.rstrip("u"), 16) for x in m.group(1).split(","))
         for m in re.finditer(r"\{(0x[0-9a-f]+u,0x[0-9a-f]+u,0x[0-9a-f]+u,0x[0-9a-f]+u|0u,0u,0u,0u)\}", c_part)]
    assert len(A) == len(C) == (1072 + 2) << 6
    return A, C


def probit_fixed(A, C, u: float) -> float:
    """The FIXED kernel's arithmetic for 0 < u < 1 (the reflection and the
    normalisation of x = 2d on the bits, segment (binade, top 6 bits),
    Tp = complement of the low 46 bits, the chains, the FMA)."""
    ub = bits(u)
    upper = ub >= 0x3FE0000000000000
    frac = ub & MANT
    eb = (ub >> 52) & 0x7FF
    S = (1 << 52) - frac if upper else ((frac | (1 << 52)) if eb else frac)
    base = 0 if upper else max(eb, 1) - 1022
    lz = 64 - (S | 1).bit_length() - 11
    Mx = S << lz
    assert 2**52 <= Mx < 2**53
    e = -1 - (base - lz)
    ec = min(max(e, -1), 1072) + 1
    idx = (ec << 6) + ((Mx >> 46) & 63)
    Tp = ~Mx & ((1 << 46) - 1)
    z = fx_row(A[idx], C[idx], Tp)
    return z if upper else -z


def fx_row(a_row, c_row, Tp: int, neg: bool = False) -> float:
    """One row of the FIXED layout at the offset Tp = Tu - 1: the chains, the
    rounding shift and bit assembly of H, and fma(+-t_u, H, a0) rounded once."""
    a0b, B0, B1, B2s = a_row
    acc = (B2s & MANT) + inner(c_row, Tp >> 15)
    acc = B1 + mulhi3(acc, Tp << 17)
    acc = B0 + mulhi3(acc, Tp << 17)
    if acc == 0:                                  # the zero rows of u = 1/2
        hbits = 0
    else:
        assert 2**61 <= acc < 2**63
        top = acc >> 62
        hbits = ((acc + (256 << top)) >> (9 + top)) + (((B2s >> 52) + top) << 52)
    tu = Fr(Tp + 1, 2**52)
    return float((-tu if neg else tu) * Fr(dbl(hbits)) + Fr(dbl(a0b)))


def normal_inputs():
    rng = np.random.default_rng(2026)
    k = rng.integers(1, 2**53, 1500, dtype=np.int64)
    uni = k.astype(np.float64) * 2.0**-53                        # 53-bit grid
    ee = rng.integers(1, 1075, 800)
    mm = rng.uniform(0.5, 1.0, 800)
    tails = np.ldexp(mm, -ee)                                     # tail stress, down to subnormal
    mirrored = 1.0 - tails[:300][tails[:300] > 2.0**-53]          # u >= 1/2 reflections
    bounds = []
    for e in (0, 1, 2, 7, 40, 300, 1000):                         # x = 2d at segment boundaries
        for j in (0, 1, 31, 62, 63):
            x = np.ldexp(1.0 + j / 64.0, -e - 1)
            bounds += [x / 2, np.nextafter(x / 2, 0.0), np.nextafter(x / 2, 1.0)]
    near_half = 0.5 + np.arange(-40, 41) * 2.0**-53
    u = np.concatenate([uni, tails, mirrored, np.array(bounds), near_half])
    return u[(u > 0) & (u < 1)]


def test_fixed_table_rows_against_the_oracle(fx_table):
    A, C = fx_table
    u = normal_inputs()
    w = oracle.probit(u)
    z = np.array([probit_fixed(A, C, float(x)) for x in u])
    zero = w == 0
    assert np.all(z[zero] == 0.0)
    r = np.abs(z[~zero] / w[~zero] - 1)
    print(f"fixed-point table rows, emulated: {len(u)} inputs, max rel {r.max():.3g}")
    assert r.max() <= 4e-15, u[~zero][np.argmax(r)]
    # symmetry is exact: x = 2d is formed identically for u and 1 - u
    pair = u[(u > 0.5) & (u < 1 - 2.0**-53)][:200]
    for x in pair:
        assert probit_fixed(A, C, float(x)) == -probit_fixed(A, C, float(1.0 - x))


@pytest.fixture(scope="module")
def exp_rows():
    """ROWS (a0 bits, B0, B1, B2 | e0) and ROWS_IN (four 32-bit words), the
    binade rows in the FIXED layout; ROW_C, the centre row (a0 bits, D0..D3,
    D4 | e0, (four 32-bit words))."""
    text = _read_text(os.path.join(CSRC, "qm_exp_fx_tables.h"))
    consts = {k: int(v) for k, v in re.findall(r"constexpr int (\w+) = (-?\d+);", text)}
    for k in ("NEAR_LO", "NEAR_HI", "POS"):
        consts[k] = int(re.search(k + r"_BITS = (0x[0-9a-fA-F]+)ull", text).group(1), 16)
    a_part = text[text.index("ROWS[NROWS] ="):text.index("ROWS_IN[NROWS] =")]
    c_part = text[text.index("ROWS_IN[NROWS] ="):text.index("ROW_C =")]
    A = [(bits(float.fromhex(m.group(1))), _int(m.group(2)) & M64, _int(m.group(3)) & M64, _int(m.group(4)) & M64)
         for m in re.finditer(r"\{(0x[0-9a-fp.+-]+|[-0-9.e+]+),([^,{}]+),([^,{}]+),([^{}]+)\}", a_part)]
    C = [tuple(int(x.rstrip("u"), 16) for x in m.group(1).split(","))
         for m in re.finditer(r"\{(0x[0-9a-f]+u,0x[0-9a-f]+u,0x[0-9a-f]+u,0x[0-9a-f]+u)\}", c_part)]
    pat = r"\{([^{},]+),(\d+)ull,(\d+)ull,(\d+)ull,(\d+)ull,(\d+)ull,\{([^}]*)\}\}"
    m = re.search(pat, text[text.index("ROW_C ="):])
    w = tuple(int(x.strip().rstrip("u"), 16) if x.strip() != "0" else 0 for x in m.group(7).split(","))
    centre = (bits(float.fromhex(m.group(1))),) + tuple(int(m.group(k)) for k in range(2, 7)) + (w,)
    n = (consts["X_EMAX"] - consts["X_EMIN"] + 1) << consts["X_K"]
    assert len(A) == len(C) == consts["NROWS"] == n and consts["X_K"] == 6
    return (A, C), centre, consts


def segtx(row, Sig: int, mlt: float) -> float:
    """One fixed-point row (Horner inner chain): fma(mlt, P(Sig 2^-64), a0)."""
    a0b, D0, D1, D2, D3, D4e, w = row
    acc = (D4e & MANT) + inner(w, Sig >> 32)
    for D in (D3, D2, D1, D0):
        assert acc < 2**62
        acc = D + mulhi3(acc, Sig)
    assert 2**59 <= acc < 2**61
    top = acc >> 60
    pm = (acc + (64 << top)) >> (7 + top)
    P = dbl(pm + (((D4e >> 52) + top) << 52))
    return float(Fr(mlt) * Fr(P) + Fr(dbl(a0b)))


def exp_fixed(rows, centre, consts, x: float):
    """The exponential -> normal kernel (None where it goes out of line:
    x < 2^-26, x >= 128, edge values): segment j (top 6 bits) of the binade
    of x, the offset t_u back from its end from the bits, the FIXED row
    arithmetic, z = -(a0 + t_u H) below 0.6875 and a0 - t_u H from there;
    |x - ln 2| < 2^-12 by the centre row in v = x - ln 2."""
    xb = bits(x)
    if xb == 0 or xb >= 0x7FF0000000000000 or xb < 0x3E50000000000000 or xb >= 0x4060000000000000:
        return None
    if consts["NEAR_LO"] <= xb < consts["NEAR_HI"]:
        v = (x - 0.69314718055994528623) - 2.3190468138462996154e-17
        t = 0.03125 - v
        tb = bits(t)
        Mt = (tb & MANT) | (1 << 52)
        st = ((tb >> 52) & 0x7FF) - 1023 + 15
        Sig = ((Mt << min(st, 63)) & (2**63 - 1)) if st >= 0 else (Mt >> -st if st > -64 else 0)
        return segtx(centre, Sig, v)
    E = (xb >> 52) - 1023
    r = ((E - consts["X_EMIN"]) << 6) + ((xb >> 46) & 63)
    Tp = ~xb & ((1 << 46) - 1)
    pos = xb >= consts["POS"]
    A, C = rows
    z = fx_row(A[r], C[r], Tp, neg=pos)
    return z if pos else -z


def test_exp_to_normal_rows_against_the_oracle(exp_rows):
    rows, centre, consts = exp_rows
    rng = np.random.default_rng(2027)
    ln2 = float(np.log(2.0))
    xs = list(rng.exponential(1.0, 2000))
    xs += list(np.exp(rng.uniform(np.log(2.0**-26), np.log(ln2), 600)))      # the X binades
    xs += list(ln2 + rng.uniform(-1 / 64, 1 / 16, 400))                       # through z = 0
    xs += list(np.exp(rng.uniform(0.0, np.log(127.9), 400)))                 # binades up to [64, 128)
    for x0 in (0.6875, 0.6953125, 0.703125, ln2, ln2 - 2.0**-12, ln2 + 2.0**-12, ln2 - 2.0**-11, ln2 + 2.0**-11,
               0.71875, 1.0, 2.0, 8.0, 64.0, 100.0):                          # the centre and binade ends
        xs += [x0, np.nextafter(x0, 0.0), np.nextafter(x0, np.inf)]
    xs = np.array([x for x in xs if x > 0])
    got = [exp_fixed(rows, centre, consts, float(x)) for x in xs]
    keep = np.array([g is not None for g in got])
    z = np.array([g for g in got if g is not None])
    w = oracle.recycle_exp(xs[keep])
    nz = w != 0
    r = np.abs(z[nz] / w[nz] - 1)
    print(f"exp -> normal rows, emulated: {int(keep.sum())} inputs, max rel {r.max():.3g}")
    assert keep.sum() > 0.98 * len(xs)
    assert r.max() <= 1e-12, xs[keep][nz][np.argmax(r)]


def _finish(acc, Ds, Sig, e0, mlt, a0b, bias):
    T16 = Sig >> 4
    for D in Ds:
        acc = (D + mulhi3(acc, Sig) - (T16 if bias else 0)) & M64
        assert 0 <= acc < 2**62
    assert 2**59 <= acc < 2**61
    top = acc >> 60
    pm = (acc + (64 << top)) >> (7 + top)
    P = dbl(pm + ((e0 + top) << 52))
    return float(Fr(mlt) * Fr(P) + Fr(dbl(a0b)))


def segts_row(r, Sig: int, mlt: float) -> float:
    """One biased row (coefficients of either sign), as the device evaluates
    it: accumulators + 2^60 (outer) and + 2^29 / + 2^25 (inner), each step
    removing the floor of what the bias contributed."""
    a0b, D0, D1, D2, D3, D4e, c01, c23 = (int(x) for x in r)
    t = Sig >> 32
    x = (((((c23 >> 32) & 0x07FFFFFF) * t) >> 32) + (c23 & 0xFFFFFFFF) - (t >> 7)) & 0xFFFFFFFF
    x = (((x * t) >> 32) + (c01 >> 32) - (t >> 3)) & 0xFFFFFFFF
    x = (((x * t) >> 32) + (c01 & 0xFFFFFFFF) - (t >> 3)) & 0xFFFFFFFF
    G = (x * t - (t << 29)) >> (c23 >> 59)                      # signed, arithmetic shift
    acc = ((D4e & MANT) + (2**60 - 2**51) + G) & M64
    return _finish(acc, (D3, D2, D1, D0), Sig, D4e >> 52, mlt, a0b, bias=True)


def inner_estrin(w, t32: int) -> int:
    """The 32-bit inner chain in Estrin form, (C_a + th C_b) + th^2 (C_c + th
    C_d), th^2 as hi32(th32 th32), and its join."""
    lo = ((w[1] * t32) >> 32) + w[0]
    hi = (((w[3] & 0x07FFFFFF) * t32) >> 32) + w[2]
    x = ((hi * ((t32 * t32) >> 32)) >> 32) + lo
    assert x < 2**32
    return (x * t32) >> (w[3] >> 27)


def fx_core(a_row, c_row, Tau: int, mlt: float, estrin: bool = False, hb: int = 61) -> float:
    """One FIXED-layout row at th = Tau 2^-64: fma(mlt, H, a0) rounded once,
    the leading bit of H(0) 2^-s0 at hb (61 for the quantile's rows, 58 for
    the Student-t rows)."""
    a0b, B0, B1, B2s = a_row
    t32 = Tau >> 32
    acc = (B2s & MANT) + (inner_estrin(c_row, t32) if estrin else inner(c_row, t32))
    acc = B1 + mulhi3(acc, Tau)
    acc = B0 + mulhi3(acc, Tau)
    assert 2**hb <= acc < 2**(hb + 2)
    top = acc >> (hb + 1)
    hbits = ((acc + ((1 << (hb - 53)) << top)) >> (hb - 52 + top)) + (((B2s >> 52) + top) << 52)
    return float(Fr(mlt) * Fr(dbl(hbits)) + Fr(dbl(a0b)))


def t_fixed(rows, z: float, estrin: bool) -> float:
    """The normal -> Student t map for |z| < 8.75: row r = floor(128 |z|)
    and Tau = (|z| 2^70) mod 2^63 from the bits, sigma = |z| - r/128 exact."""
    A, C = rows
    a = abs(z)
    ab = bits(a)
    E = (ab >> 52) - 1023
    M = (ab & MANT) | (1 << 52)
    r = 0 if E + 7 < 0 else M >> (52 - (E + 7))
    lr = (r | 1).bit_length() - 1
    zsb = 0 if r == 0 else ((lr - 7 + 1023) << 52) | ((r << (52 - lr)) & MANT)
    sig = a - dbl(zsb)
    sh = E + 18
    Tau = ((M << sh) & (2**63 - 1)) if sh >= 0 else (M >> -sh if sh > -64 else 0)
    a_row = tuple(int(x) for x in A[r])
    c_row = tuple(int(x) for x in C[r])
    t = fx_core(a_row, c_row, Tau, sig, estrin, hb=58)
    return t if z >= 0 else -t


@pytest.mark.parametrize("nu", [0.75, 1.0, 2.7, 4.0, 30.0, 100.0])
def test_student_t_rows_against_the_oracle(nu):
    import paper_0901_0638_gb300 as qm
    rows = qm.qm_t_rows_build(nu)
    rng = np.random.default_rng(int(nu * 100))
    z = np.concatenate([rng.standard_normal(400) * 2.5, rng.uniform(-8.74, 8.74, 200),
                        np.arange(1, 1120) / 128.0, np.arange(1, 1120) / 128.0 - 2.0**-40,
                        [1e-300, 2.0**-20, -3e-9, 8.75 - 2.0**-40]])
    z = z[np.abs(z) < 8.75]
    w = oracle.recycle_t(nu, z)
    for estrin in (False, True):
        got = np.array([t_fixed(rows, float(x), estrin) for x in z])
        r = np.abs(got / w - 1)
        print(f"Student t nu={nu} rows ({'Estrin' if estrin else 'Horner'}): max rel {r.max():.3g}")
        assert r.max() <= 1e-12, (estrin, z[np.argmax(r)])


@pytest.mark.parametrize("abd", [(1.3, 0.4, 0.7), (2.0, -1.5, 0.05)])
def test_hyperbolic_biased_rows_against_the_oracle(abd):
    import paper_0901_0638_gb300 as qm
    from oracle.hyperbolic import Hyperbolic, recycle_hyperbolic
    a, b, d = abd
    R, L, e_max = qm.qm_hyp_rows_build(a, b, d)
    o = Hyperbolic(a, b, d)
    rng = np.random.default_rng(7)
    side = rng.random(160) < o.p_plus
    v = np.where(side, rng.exponential(1 / (a - b), 160), -rng.exponential(1 / (a + b), 160))
    v = np.concatenate([v, [2.0**-29, -2.0**-29 * 1.5, 1e-6, -1e-3, 0.75, -0.75]])
    got = []
    for x in v:
        ab = bits(abs(float(x)))
        E = (ab >> 52) - 1023
        rows = R if x > 0 else L
        assert qm.QM_HYP_E_MIN <= E <= e_max[0 if x > 0 else 1]
        low = ab & ((1 << 47) - 1)
        sig = abs(float(x)) - dbl(ab - low)
        m = segts_row(rows[32 * (E - qm.QM_HYP_E_MIN) + ((ab >> 47) & 31)], low << 16, sig)
        got.append(m if x > 0 else -m)
    w = recycle_hyperbolic(a, b, d, v)
    r = np.abs(np.array(got) / w - 1)
    print(f"hyperbolic {abd} biased rows: max rel {r.max():.3g}")
    assert r.max() <= 1e-12, v[np.argmax(r)]


def _generated(fn, *args):
    """Run one row generator at its own mpmath precision, restoring the
    caller's afterwards."""
    import mpmath as mp
    with mp.workprec(mp.mp.prec):
        return fn(*args)


def _row_fields(q):
    """The device words of one FIXED-layout row from a generator's fields."""
    a = (bits(float(q["a0"])), q["B"][0] & M64, q["B"][1] & M64, ((q["e0"] << 52) | q["B"][2]) & M64)
    c = tuple(q["C"][:3]) + (q["C"][3] | (q["sh"] << 27),)
    return a, c


def test_fixed_table_rows_are_what_their_generator_writes(fx_table):
    """Rows of csrc/qm_fx_tables.h regenerated one by one from
    fit/gen_fx_tables.py (the u = 1/2 binade, the middle of the main
    binades, the first deep binade, the last binade) equal the committed
    words: the table is the generator's output and nothing else."""
    pytest.importorskip("mpmath")
    from paper_0901_0638_gb300.fit import gen_fx_tables as G
    A, C = fx_table
    for e, j in ((0, 0), (0, 63), (17, 31), (63, 63), (64, 0), (500, 17), (G.E_LAST, 63)):
        e_, j_, q, worst = _generated(G.job, (e, j))
        row = G.seg_index(e, j) + (1 << G.K_MAIN)               # after the zero rows of u = 1/2
        assert (e_, j_) == (e, j) and worst < 4e-16, (e, j, worst)
        assert (A[row], C[row]) == _row_fields(q), (e, j)


def test_exp_to_normal_rows_are_what_their_generator_writes(exp_rows):
    """Rows of csrc/qm_exp_fx_tables.h regenerated from
    fit/gen_exp_fx_tables.py -- binade rows on both sides of ln 2 (the
    segment that holds it included) and the centre row -- equal the
    committed words."""
    pytest.importorskip("mpmath")
    from paper_0901_0638_gb300.fit import gen_exp_fx_tables as G
    (A, C), centre, consts = exp_rows
    cells = [(G.X_EMIN, 0), (-8, 40), (-1, 0), (-1, 24), (-1, 25), (0, 7), (G.X_EMAX, 63)]
    for E, j in cells:
        E_, j_, side, q, worst = _generated(G.binade_row, (E, j))
        row = ((E - consts["X_EMIN"]) << consts["X_K"]) + j
        assert (E_, j_) == (E, j) and side == ("pos" if E >= -1 and (E > -1 or j >= 24) else "neg")
        assert worst < 2e-15, (E, j, worst)
        assert (A[row], C[row]) == _row_fields(q), (E, j)
    a0, D, f, e0, worst = _generated(G.centre_row)
    assert worst < 1e-13
    assert centre == (bits(a0), D[0], D[1], D[2], D[3], (e0 << 52) | D[4], tuple(f))
