"""Normal -> Student t tables for any real nu, built on the host (no GPU).

qm_t_table_build returns the segment expansions and the tail series that
qm_recycle uploads for an untabulated nu.  They are checked here against
values the paper fixes (Sec. 3.2: Q'(0) = gamma and the closed forms of
c_1, c_2; Sec. 3.3: R'(0) = -(nu+1)/(2(nu+2)); the tail constant c) and,
evaluated in numpy, against the CPU oracle's incomplete-beta quantile
within the 1e-12 relative tolerance of the recycled Student t.
"""
import math

import numpy as np
import pytest
from scipy import special

import oracle
import paper_0901_0638_gb300 as qm


def _read_text(path):
    with open(path) as fh:
        return fh.read()


NUS = [0.75, 1.0, 1.5, 2.5, 4.0, 6.3, 17.0, 50.0, 100.0]


def gamma_c0(nu):
    """Q'(0) = gamma = sqrt(nu/2) Gamma(nu/2) / Gamma((nu+1)/2) (Sec. 3.1), 30 digits."""
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    return float(mp.sqrt(mp.mpf(nu) / 2) * mp.gamma(mp.mpf(nu) / 2) / mp.gamma((mp.mpf(nu) + 1) / 2))


def evaluate(seg, tail, z):
    """The device's evaluation order in float64 (segments, then the tail)."""
    z = np.asarray(z, dtype=np.float64)
    a = np.abs(z)
    out = np.empty_like(a)
    c = a < 8.75
    j = np.floor(a[c] * 32).astype(int)
    zc = np.where(j == 0, 0.0, (2 * j + 1) / 64.0)
    s = a[c] - zc
    acc = np.zeros_like(s)
    for k in range(9, -1, -1):
        acc = acc * s + seg[j, k]
    out[c] = acc
    t = ~c
    nu, lk, deg = tail[0], tail[1], int(tail[2])
    lw = lk + special.log_ndtr(-a[t])
    y = np.exp(2.0 / nu * lw)
    r = np.zeros_like(y)
    for k in range(deg, -1, -1):
        r = r * y + tail[3 + k]
    with np.errstate(over="ignore"):                  # inf where the t quantile overflows a double
        out[t] = math.sqrt(nu) * np.exp(-lw / nu) * r
    return np.copysign(out, z)


@pytest.mark.parametrize("nu", NUS)
def test_central_series_matches_the_paper(nu):
    seg, tail = qm.qm_t_table_build(nu)
    g = gamma_c0(nu)
    c = seg[0]
    # odd series about z = 0 (Sec. 3.2)
    assert np.all(c[0::2] == 0.0) or np.max(np.abs(c[0::2])) < 1e-16 * g
    assert abs(c[1] / g - 1) < 1e-15
    c1 = ((nu + 1) * g**3 - nu * g) / (6 * nu)
    c2 = ((7 * nu**2 + 8 * nu + 1) * g**5 - (10 * nu**2 + 10 * nu) * g**3 + 3 * nu**2 * g) / (120 * nu**2)
    assert abs(c[3] - c1) <= 1e-14 * max(abs(c1), g)
    assert abs(c[5] - c2) <= 1e-13 * max(abs(c2), g)


@pytest.mark.parametrize("nu", NUS)
def test_tail_series_matches_the_paper(nu):
    _, tail = qm.qm_t_table_build(nu)
    assert tail[0] == nu and int(tail[2]) == qm.QM_T_TAIL_TERMS - 1
    assert tail[3] == 1.0
    assert abs(tail[4] + (nu + 1) / (2 * (nu + 2))) < 1e-15
    # c = sqrt(nu) kappa^{-1/nu} with kappa = nu sqrt(pi) Gamma(nu/2) / Gamma((nu+1)/2)
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 30
    n = mp.mpf(nu)
    log_kappa = float(mp.log(n * mp.sqrt(mp.pi) * mp.gamma(n / 2) / mp.gamma((n + 1) / 2)))
    assert abs(tail[1] - log_kappa) < 4e-16 * max(1.0, abs(log_kappa))


@pytest.mark.parametrize("nu", NUS)
def test_expansions_against_the_oracle(nu):
    seg, tail = qm.qm_t_table_build(nu)
    rng = np.random.default_rng(int(nu * 1000))
    z = np.concatenate([rng.uniform(0, 8.75, 4000), np.arange(0, 280) / 32.0, (np.arange(280) + 0.999) / 32,
                        rng.uniform(8.75, 38.0, 300), [1e-300, 1e-12, 8.75, 37.5], -rng.uniform(0, 10, 200)])
    t = evaluate(seg, tail, z)
    w = oracle.recycle_t(nu, z)
    ok = np.isfinite(w) & (w != 0)
    rel = np.abs(t[ok] / w[ok] - 1)
    assert rel.max() <= 1e-12, (nu, z[ok][np.argmax(rel)], rel.max())


def test_closed_forms_nu_1_and_2():
    # nu = 1: t = tan(pi (Phi(z) - 1/2)); nu = 2: t = (2u - 1)/sqrt(2 u (1 - u))
    z = np.linspace(-6, 6, 241)
    u = special.ndtr(z)
    seg, tail = qm.qm_t_table_build(1.0)
    t1 = evaluate(seg, tail, z)
    ref1 = np.tan(np.pi * (u - 0.5))
    m = np.abs(z) < 3
    assert np.allclose(t1[m], ref1[m], rtol=1e-12, atol=0)
    seg, tail = qm.qm_t_table_build(2.0)
    t2 = evaluate(seg, tail, z)
    ref2 = (2 * u - 1) / np.sqrt(2 * u * (1 - u))
    assert np.allclose(t2[m], ref2[m], rtol=1e-12, atol=0)


def test_out_of_range_nu_is_rejected():
    for nu in (0.5, 0.25, 100.5, 0.0, -1.0, float("nan"), float("inf")):
        for build in (qm.qm_t_table_build, qm.qm_t_rows_build):
            with pytest.raises(qm.QMError) as e:
                build(nu)
            assert e.value.status == qm.QM_ERR_UNSUPPORTED, (build.__name__, nu)


def test_offline_t_tables_are_what_their_generator_writes():
    """Segments and tail series of csrc/qm_t_tables.h (the tabulated nu)
    regenerated from fit/gen_t_tables.py equal the committed literals: the
    first, a middle and the last segment of three nu, and every tail row."""
    mp = pytest.importorskip("mpmath")
    import os
    import re
    from paper_0901_0638_gb300.fit import gen_t_tables as G
    text = _read_text(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                             "paper_0901_0638_gb300", "csrc", "qm_t_tables.h"))
    body = text[text.index("SEG_T[NNU * NSEG] = {"):text.index("T_KAPPA")]
    rows = re.findall(r"\{\{([^}]*)\},\{([^}]*)\},0\.0f\}", body)
    assert len(rows) == len(G.NU_SET) * G.NSEG
    tails = re.findall(r"^  \{([^{}]*)\},$", text[text.index("T_TAIL["):], flags=re.M)
    assert len(tails) == len(G.NU_SET)
    with mp.workprec(mp.mp.prec):
        for i, nu in enumerate(G.NU_SET):
            if nu in (1, 4, 30):
                for j in (0, G.NSEG // 2, G.NSEG - 1):
                    _, _, b, _ = G.seg((nu, j))
                    d, f = rows[i * G.NSEG + j]
                    assert d == ",".join(G.hexd(x) for x in b[:5]), (nu, j)
                    assert f == ",".join(G.hexf(x) for x in b[5:10]), (nu, j)
            _, R, worst, _ = G.tail_fit(nu)
            assert tails[i] == ",".join(G.hexd(c) for c in R), nu
