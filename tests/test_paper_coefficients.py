"""The paper's printed rational approximations, as the library stores them
for QM_VAR_PAPER_EXACT (csrc/qm_paper_coeffs.h), against the theoretical
accuracy the paper states for them, evaluated in 50-digit mpmath with the
printed decimal digits:

  (5,6)   exponential coordinate, v in [0, 25]:   < 2.98e-8   (Sec. 6.1, Appendix A)
  (13,13) exponential coordinate, v in [0, 42]:   < 5.4e-17   (Sec. 7.2, Appendix B)
  (14,15) scaled t_2 coordinate,  v in [0, 15.5]: < 5.55e-17  (Sec. 7.3, Appendix C)

The exact maps are Q(v) = Phi^{-1}(1 - e^{-v}/2) = sqrt2 erfinv(1 - e^{-v}) and,
for t_2, Phi^{-1}(u) at u = 1/2 + v / (2 sqrt(1 + v^2)), i.e.
sqrt2 erfinv(v / sqrt(1 + v^2)).  A minimax rational equioscillates, so its
largest error on a dense grid lies just below the stated bound; a wrong digit,
sign, order or degree in a stored coefficient moves it far from there.
"""
import os
import re

import pytest


def _read_text(path):
    with open(path) as fh:
        return fh.read()


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "paper_0901_0638_gb300", "csrc", "qm_paper_coeffs.h")


def stored_tables():
    src = _read_text(HEADER)
    out = {}
    for name in ("A_P", "A_Q", "B_P", "B_Q", "C_P", "C_Q"):
        m = re.search(name + r"\[\w+\]\s*=\s*\{(.*?)\};", src, re.S)
        assert m, name
        out[name] = re.findall(r"[0-9][0-9.]*(?:e[-+]?[0-9]+)?", m.group(1))
    return out


def max_rel_error(mp, p, q, exact, vmax, npts=2400):
    """Largest |v p(v)/q(v) / exact(v) - 1| over a Chebyshev-clustered grid
    of (0, vmax], each local maximum refined by golden-section search."""
    P = [mp.mpf(c) for c in p]
    Q = [mp.mpf(c) for c in q]

    def err(v):
        v = mp.mpf(v)
        return abs(v * mp.polyval(P[::-1], v) / mp.polyval(Q[::-1], v) / exact(v) - 1)

    vs = [vmax * (1 - mp.cos(mp.pi * (k + 0.5) / npts)) / 2 for k in range(npts)] + [mp.mpf(vmax)]
    es = [err(v) for v in vs]
    best = max(es)
    for k in range(1, len(vs) - 1):
        if es[k] >= es[k - 1] and es[k] >= es[k + 1] and es[k] > best / 2:
            lo, hi = vs[k - 1], vs[k + 1]
            for _ in range(30):
                a, b = lo + (hi - lo) * 0.382, lo + (hi - lo) * 0.618
                if err(a) > err(b):
                    hi = b
                else:
                    lo = a
            best = max(best, err((lo + hi) / 2))
    return float(best)


@pytest.mark.parametrize("table,vmax,bound", [("A", 25, 2.98e-8), ("B", 42, 5.4e-17), ("C", 15.5, 5.55e-17)])
def test_printed_rationals_reach_the_stated_bounds(table, vmax, bound):
    mp = pytest.importorskip("mpmath")
    t = stored_tables()
    p, q = t[table + "_P"], t[table + "_Q"]
    assert (len(p), len(q)) == {"A": (6, 7), "B": (14, 14), "C": (15, 16)}[table]
    with mp.workdps(50):
        if table == "C":
            exact = lambda v: mp.sqrt(2) * mp.erfinv(v / mp.sqrt(1 + v * v))
        else:
            exact = lambda v: mp.sqrt(2) * mp.erfinv(-mp.expm1(-v))
        e = max_rel_error(mp, p, q, exact, vmax)
    print(f"({table}) max relative error on [0, {vmax}]: {e:.4g} (stated < {bound:g})")
    assert bound / 2 < e < bound
