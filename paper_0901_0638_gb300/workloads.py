"""Seeded synthetic inputs shaped like the paper's workloads.

This module is the one piece shared by the tests, the bench and the oracle
checks.  It holds no arithmetic of the quantile method: only counter-based
random bits (Philox4x32-10, Salmon et al. SC'11) and the recipes that turn them
into the input arrays.  Everything is written with torch integer/float tensor
operations so the same call gives bit-identical results on the CPU and on a
GPU (the 32x32-bit products are split into 16-bit halves so that no int64
product overflows).

Stream layout (shared with the library's fused sampler): word ``i`` of the
stream with seed ``s`` is output word ``i mod 4`` of Philox4x32-10 with key
``(s mod 2^32, s >> 32)`` and 128-bit counter ``floor(i/4)`` spread
little-endian over the four counter words.
"""
from __future__ import annotations

import math

import torch

_M0, _M1 = 0xD2511F53, 0xCD9E8D57
_W0, _W1 = 0x9E3779B9, 0xBB67AE85
_MASK32 = 0xFFFFFFFF


def _mulhilo(a: torch.Tensor, m: int):
    ml, mh = m & 0xFFFF, m >> 16
    t1 = a * ml            # < 2^48
    t2 = a * mh            # < 2^48
    lo = (((t2 & 0xFFFF) << 16) + t1) & _MASK32
    hi = (t2 + (t1 >> 16)) >> 16
    return hi, lo


def philox_blocks(seed: int, c0: torch.Tensor, c1=None, c2=None, c3=None):
    """Philox4x32-10 of counters (c0, c1, c2, c3) (int64 tensors holding
    uint32 values) under key (seed lo, seed hi).  Returns four int64 tensors."""
    z = torch.zeros_like(c0)
    x0 = c0 & _MASK32
    x1 = (c1 if c1 is not None else z) & _MASK32
    x2 = (c2 if c2 is not None else z) & _MASK32
    x3 = (c3 if c3 is not None else z) & _MASK32
    k0, k1 = seed & _MASK32, (seed >> 32) & _MASK32
    for _ in range(10):
        hi0, lo0 = _mulhilo(x0, _M0)
        hi1, lo1 = _mulhilo(x2, _M1)
        x0, x1, x2, x3 = hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0
        k0 = (k0 + _W0) & _MASK32
        k1 = (k1 + _W1) & _MASK32
    return x0, x1, x2, x3


def philox_words(seed: int, first: int, n: int, device="cpu") -> torch.Tensor:
    """Words first..first+n-1 of the stream (int64 tensor of uint32 values)."""
    idx = torch.arange(first, first + n, dtype=torch.int64, device=device)
    blk = idx >> 2
    w = philox_blocks(seed, blk & _MASK32, blk >> 32)
    sel = idx & 3
    out = torch.where(sel == 0, w[0], w[1])
    out = torch.where(sel == 2, w[2], out)
    out = torch.where(sel == 3, w[3], out)
    return out


# ---------------------------------------------------------------------------
# FP32 normal quantile on 2^20 uniforms u_i = (k + 0.5) / 2^24, k the top 24
# bits of Philox word i (seed 1).
# ---------------------------------------------------------------------------
def uniform24(seed: int, n: int, first: int = 0, device="cpu"):
    """Returns (k, u32): k = word >> 8 (int64) and u32 = fl32((k + 0.5)/2^24)
    rounded to nearest even (k = 2^24 - 1 gives exactly 1.0f)."""
    k = philox_words(seed, first, n, device) >> 8
    u = ((k.to(torch.float64) + 0.5) * 2.0 ** -24).to(torch.float32)
    return k, u


# ---------------------------------------------------------------------------
# FP64 normal quantile on n doubles (seed 2): 90 % uniform k 2^-53 with
# k in [1, 2^53 - 1]; 10 % tail stress 2^-e m, e uniform in [1, 990], m uniform
# in [1/2, 1), each mirrored to fl(1 - u) with probability 1/2.  Element i
# draws the four words of Philox block (i lo, i hi, 0, 0).
# ---------------------------------------------------------------------------
STRESS_THRESHOLD = 429496730  # round(0.1 * 2^32)


def mixture_f64(seed: int, n: int, first: int = 0, device="cpu") -> torch.Tensor:
    idx = torch.arange(first, first + n, dtype=torch.int64, device=device)
    w0, w1, w2, w3 = philox_blocks(seed, idx & _MASK32, idx >> 32)
    stress = w0 < STRESS_THRESHOLD
    k53 = ((w1 >> 11) << 32) | w2
    k53 = torch.clamp(k53, min=1)
    u_uni = k53.to(torch.float64) * 2.0 ** -53
    e = 1 + ((w1 * 990) >> 32)
    frac = ((w2 & 0xFFFFF) << 32) | w3
    m = (frac + (1 << 52)).to(torch.float64) * 2.0 ** -53
    u_st = torch.ldexp(m, -e.to(torch.float64))
    mirror = (w1 & 1) == 1
    u_st = torch.where(mirror, 1.0 - u_st, u_st)
    return torch.where(stress, u_st, u_uni)


# ---------------------------------------------------------------------------
# Samplers for the recycling maps (53-bit uniforms in (0, 1)).
# ---------------------------------------------------------------------------
def uniform53(seed: int, n: int, first: int = 0, stream: int = 0,
              device="cpu") -> torch.Tensor:
    """u = (k + 1/2) 2^-53 from words (2j, 2j+1) of block (j, stream): open
    interval, never 0 or 1."""
    j = torch.arange(first, first + n, dtype=torch.int64, device=device)
    w0, w1, _, _ = philox_blocks(seed, j & _MASK32, j >> 32,
                                 torch.full_like(j, stream & _MASK32))
    k = ((w0 >> 11) << 32) | w1
    return (k.to(torch.float64) + 0.5) * 2.0 ** -53


def normal_box_muller(seed: int, n: int, first: int = 0, stream: int = 0,
                      device="cpu") -> torch.Tensor:
    """Standard normals by Box-Muller, z = sqrt(-2 ln u1) cos(2 pi u2)."""
    u1 = uniform53(seed, n, first, 2 * stream, device)
    u2 = uniform53(seed, n, first, 2 * stream + 1, device)
    return torch.sqrt(-2.0 * torch.log(u1)) * torch.cos(2.0 * math.pi * u2)


def exponential(seed: int, n: int, first: int = 0, stream: int = 0,
                device="cpu") -> torch.Tensor:
    """Exp(1) samples x = -ln u."""
    return -torch.log(uniform53(seed, n, first, 2 * stream, device))


# ---------------------------------------------------------------------------
# Ragged recycling batch: segments with lengths log-uniform in [2^lo, 2^hi].
# Target code: 0..7 -> Student t with NU_SET[code], 8 -> exponential->normal.
# ---------------------------------------------------------------------------
NU_SET = (1.0, 2.0, 3.0, 4.0, 5.0, 8.0, 10.0, 30.0)


def ragged_segments(seed: int = 4, nseg: int = 256, lo: int = 10, hi: int = 24):
    w = philox_words(seed, 0, 2 * nseg)
    r = w[0::2].to(torch.float64) * 2.0 ** -32
    lens = torch.floor(2.0 ** (lo + (hi - lo) * r)).to(torch.int64)
    targets = (w[1::2] * 9) >> 32
    return lens.tolist(), targets.tolist()


# ---------------------------------------------------------------------------
# Serving trace: Poisson arrivals, log-uniform sizes, mixed targets.
# ---------------------------------------------------------------------------
def serving_trace(seed: int = 5, rate: float = 2e4, seconds: float = 10.0,
                  lo: int = 8, hi: int = 24, max_requests=None):
    """Returns a list of dicts {t_arrival, n, kind, nu, key}.  kind: 0 normal
    FP32, 1 normal FP64, 2 Student t (nu from NU_SET), 3 exponential->normal."""
    cap = int(rate * seconds * 1.5) + 64
    w = philox_words(seed, 0, 4 * cap).view(-1, 4)
    u = (w[:, 0].to(torch.float64) + 0.5) * 2.0 ** -32
    gaps = -torch.log(u) / rate
    t = torch.cumsum(gaps, 0)
    ns = torch.floor(2.0 ** (lo + (hi - lo) * w[:, 1].to(torch.float64) * 2.0 ** -32))
    kinds = (w[:, 2] * 4) >> 32
    nus = (w[:, 3] * 8) >> 32
    out = []
    for i in range(cap):
        ti = float(t[i])
        if ti > seconds:
            break
        if max_requests is not None and i >= max_requests:
            break
        out.append({"t_arrival": ti, "n": int(ns[i]), "kind": int(kinds[i]),
                    "nu": NU_SET[int(nus[i])], "key": (seed << 32) + i + 1})
    return out
