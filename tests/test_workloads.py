"""The seeded input generators: bit-identical to the oracle's Philox stream
and to the recipes stated in their docstrings."""
import numpy as np
import torch

import oracle
from paper_0901_0638_gb300 import workloads as W


def test_philox_words_match_oracle_stream():
    for seed, first in [(1, 0), (3, 12345), (2**40 + 9, 4 * (2**32 - 2))]:
        a = W.philox_words(seed, first, 37).numpy().astype(np.uint32)
        b = oracle.philox_stream(seed, first, 37)
        assert np.array_equal(a, b)


def test_uniform24_rounding():
    k, u = W.uniform24(1, 4096)
    assert k.min() >= 0 and k.max() < 2**24
    exact = (k.double() + 0.5) * 2.0**-24
    assert torch.equal(u, exact.float())
    # the top grid point rounds to 1.0f
    top = torch.tensor([2**24 - 1], dtype=torch.float64)
    assert float(((top + 0.5) * 2.0**-24).float()) == 1.0


def test_mixture_recipe():
    u = W.mixture_f64(2, 1 << 16)
    assert torch.all((u > 0) & (u <= 1))
    frac_small = float((u < 2.0**-60).double().mean())
    frac_one = float((u == 1.0).double().mean())
    # ~10% stress x P(e > 60)~0.94 x 1/2 unmirrored; ~4.7% become exactly 1.0
    assert 0.04 < frac_small < 0.055 and 0.04 < frac_one < 0.055
    assert torch.equal(u[:1000], W.mixture_f64(2, 1000))
    assert torch.equal(u[500:600], W.mixture_f64(2, 100, first=500))


def test_ragged_segments_and_trace():
    lens, tg = W.ragged_segments(4, 256)
    assert len(lens) == 256 and min(lens) >= 2**10 and max(lens) <= 2**24
    assert set(tg) <= set(range(9)) and len(set(tg)) == 9
    tr = W.serving_trace(5, rate=2e4, seconds=0.05)
    assert 800 < len(tr) < 1200
    assert all(2**8 <= r["n"] <= 2**24 for r in tr)
