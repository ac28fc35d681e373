"""GPU parity of the exponential -> hyperbolic recycling map (Sec. 8.1)
against the CPU oracle (quadrature + Brent), 1e-12 relative; edge values
exact; in-place and ragged sizes."""
import math

import numpy as np
import pytest
import torch

import paper_0901_0638_gb300 as qm
from oracle.hyperbolic import Hyperbolic, recycle_hyperbolic
from tests.gpu_util import rel_err

pytestmark = pytest.mark.gpu
DEV = "cuda"
PARAMS = [(1.0, 0.0, 1.0), (1.3, 0.4, 0.7), (2.0, -1.5, 0.05), (0.5, 0.2, 5.0), (1.0, 0.9, 2.0)]


def base_samples(a, b, p_plus, n, seed):
    rng = np.random.default_rng(seed)
    side = rng.random(n) < p_plus
    v = np.where(side, rng.exponential(1 / (a - b), n), -rng.exponential(1 / (a + b), n))
    mags = np.array([5e-324, 1e-300, 1e-20, 2.0**-30, 2.0**-29 * 1.5, 1e-9, 1e-3, 0.25, 1.0, 5.0, 30.0, 120.0])
    return np.concatenate([v, mags, -mags, [700 / (a - b), -700 / (a + b)]])


@pytest.mark.parametrize("a,b,d", PARAMS)
def test_hyperbolic_map_vs_oracle(a, b, d):
    h = qm.Hyperbolic(a, b, d)
    o = Hyperbolic(a, b, d)
    info = h.info()
    assert abs(info["p_plus"] / o.p_plus - 1) < 1e-14
    v = base_samples(a, b, o.p_plus, 3000, seed=int(1000 * abs(a + 3 * b + 7 * d)))
    vd = torch.from_numpy(v).to(DEV)
    xd = torch.empty_like(vd)
    h.recycle(vd, xd)
    torch.cuda.synchronize()
    x = xd.cpu().numpy()
    w = recycle_hyperbolic(a, b, d, v)
    normal = np.abs(w) >= 1e-290
    r = rel_err(x[normal], w[normal])
    print(f"hyperbolic {(a, b, d)}: max rel {r.max():.3g}")
    assert r.max() <= 1e-12, (v[normal][np.argmax(r)], r.max())
    # |v| this small: Q is linear, Q(v) = Q'(0+-) v (the oracle's bracketing
    # tolerance cannot resolve such outputs), to within one subnormal step.
    # The slopes from the closed form of Sec. 8.1, not from the library:
    # Q'(0+-) = f_0(0+-) / f(0) = p_+- (alpha -+ beta) Z e^{alpha delta},
    # Z = 2 alpha delta K_1(delta gamma) / gamma
    from scipy import special
    g = math.sqrt(a * a - b * b)
    zf = 2 * a * d * special.kv(1, d * g) / g * math.exp(a * d)
    s_plus, s_minus = o.p_plus * (a - b) * zf, o.p_minus * (a + b) * zf
    assert abs(info["slope_plus"] / s_plus - 1) < 1e-13 and abs(info["slope_minus"] / s_minus - 1) < 1e-13
    tiny = ~normal & (v != 0)
    slope = np.where(v[tiny] > 0, s_plus, s_minus)
    # (the library's slope, from its own quadrature, agrees with the closed
    # form to ~1e-15, within 4e-15 asserted above via 1e-13)
    assert np.all(np.abs(x[tiny] - slope * v[tiny]) <= 5e-324 + 4e-15 * np.abs(slope * v[tiny]))
    assert np.all(np.sign(x) == np.sign(v))
    h.close()


def test_hyperbolic_edges_inplace_ragged():
    h = qm.Hyperbolic(1.3, 0.4, 0.7)
    edge = torch.tensor([0.0, -0.0, math.inf, -math.inf, math.nan], dtype=torch.float64, device=DEV)
    out = torch.empty_like(edge)
    h.recycle(edge, out)
    torch.cuda.synchronize()
    e = out.cpu().numpy()
    assert e[0] == 0.0 and math.copysign(1, e[1]) == -1.0 and e[2] == math.inf and e[3] == -math.inf
    assert math.isnan(e[4])
    for n in (1, 2, 3, 255, 257, 4099):
        v = torch.from_numpy(base_samples(1.3, 0.4, 0.5, n, seed=n)[:n]).to(DEV)
        ref = torch.empty_like(v)
        h.recycle(v, ref)
        inplace = v.clone()
        h.recycle(inplace, inplace)
        torch.cuda.synchronize()
        assert torch.equal(ref, inplace)
    h.close()


def test_hyperbolic_argument_errors():
    with pytest.raises(qm.QMError) as e:
        qm.Hyperbolic(1.0, 1.5, 1.0)
    assert e.value.status == qm.QM_ERR_INVALID
    with pytest.raises(qm.QMError) as e:
        qm.Hyperbolic(1.0, 0.0, 1e-7)
    assert e.value.status == qm.QM_ERR_UNSUPPORTED
