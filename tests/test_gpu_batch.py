"""Ragged batch (one persistent graph launch over a segment table) against
the oracle, against per-segment launches, and alone vs in the batch."""
import numpy as np
import pytest
import torch

import oracle
import paper_0901_0638_gb300 as qm
from paper_0901_0638_gb300 import workloads as W
from tests.gpu_util import f64_violations

pytestmark = pytest.mark.gpu
DEV = "cuda"


def make_batch(lens, targets, seed=4, device=DEV):
    segs, ins, outs = [], [], []
    for j, (n, tg) in enumerate(zip(lens, targets)):
        if tg == 8:
            x = W.exponential(seed, n, 0, j + 1, device)
            segs.append((qm.QM_DIST_EXPONENTIAL, qm.QM_DIST_NORMAL, 0.0))
        else:
            x = W.normal_box_muller(seed, n, 0, j + 1, device)
            segs.append((qm.QM_DIST_NORMAL, qm.QM_DIST_STUDENT_T, W.NU_SET[tg]))
        ins.append(x)
        outs.append(torch.full_like(x, float("nan")))
    spec = [(s, d, nu, i, o) for (s, d, nu), i, o in zip(segs, ins, outs)]
    return spec, ins, outs


def oracle_of(spec_entry, x):
    src, dst, nu, _, _ = spec_entry
    return oracle.recycle_exp(x) if src == qm.QM_DIST_EXPONENTIAL else oracle.recycle_t(nu, x)


def test_batch_small_ragged_vs_oracle_and_alone():
    rng = np.random.default_rng(4)
    lens = [int(2 ** rng.uniform(10, 15)) for _ in range(48)] + [1, 2, 3, 257]
    targets = [k % 9 for k in range(len(lens))]
    spec, ins, outs = make_batch(lens, targets)
    b = qm.Batch(spec, tuning=(256, 2, 0))
    b.run()
    torch.cuda.synchronize()
    for e, x, o in zip(spec, ins, outs):
        w = oracle_of(e, x.cpu().numpy())
        assert not f64_violations(o.cpu().numpy(), w, 1e-12).any(), e[:3]
        # the same segment alone through qm_recycle: bit-identical (same form)
        alone = torch.empty_like(x)
        qm.qm_recycle(e[0], e[1], x, alone, nu=e[2] if e[1] == qm.QM_DIST_STUDENT_T else None)
        torch.cuda.synchronize()
        assert torch.equal(alone, o), e[:3]
    # replaying the graph and the per-segment launches give the same bits
    saved = [o.clone() for o in outs]
    for o in outs:
        o.fill_(float("nan"))
    b.run_separate()
    torch.cuda.synchronize()
    assert all(torch.equal(a, c) for a, c in zip(saved, outs))
    b.close()


def test_batch_with_untabulated_nu():
    """Segments with any real nu (run-time tables) next to tabulated ones."""
    lens = [3000, 1025, 77, 4096, 513]
    nus = [2.7, 13.0, 0.8, 4.0, 2.7]
    segs, ins, outs = [], [], []
    for j, (n, nu) in enumerate(zip(lens, nus)):
        x = W.normal_box_muller(11, n, 0, j + 1, DEV)
        segs.append((qm.QM_DIST_NORMAL, qm.QM_DIST_STUDENT_T, nu, x, torch.full_like(x, float("nan"))))
    for tuning in ((256, 2, 0), (128, 4, 1)):
        b = qm.Batch(segs, tuning=tuning)
        b.run()
        torch.cuda.synchronize()
        for (src, dst, nu, x, o) in segs:
            w = oracle.recycle_t(nu, x.cpu().numpy())
            assert not f64_violations(o.cpu().numpy(), w, 1e-12).any(), (tuning, nu)
            if tuning[2] == 0:
                alone = torch.empty_like(x)
                qm.qm_recycle(src, dst, x, alone, nu=nu)
                torch.cuda.synchronize()
                assert torch.equal(alone, o), nu
        b.close()


def test_batch_tuning_candidates_and_autotuner(tmp_path, monkeypatch):
    monkeypatch.setenv("QM_TUNE_CACHE", str(tmp_path / "tune.txt"))
    rng = np.random.default_rng(8)
    lens = [int(2 ** rng.uniform(10, 16)) for _ in range(24)]
    targets = [k % 9 for k in range(len(lens))]
    spec, ins, outs = make_batch(lens, targets, seed=5)
    b = qm.Batch(spec, tuning=(128, 1, 1))
    for t in [(128, 1, 1), (512, 4, 0), (256, 2, 1)]:
        b.set_tuning(t)
        b.run()
        torch.cuda.synchronize()
        for e, x, o in zip(spec, ins, outs):
            w = oracle_of(e, x.cpu().numpy())
            assert not f64_violations(o.cpu().numpy(), w, 1e-12).any(), (t, e[:3])
    best = b.tune(reps=2)
    assert best in [(bl, ep, es) for bl in (128, 256, 512) for ep in (1, 2, 4) for es in (0, 1)]
    assert (tmp_path / "tune.txt").read_text().strip().endswith(" ".join(map(str, best)))
    b.close()
    # a new batch with the same signature picks the cached tuning
    b2 = qm.Batch(spec)
    assert b2.tuning() == best
    b2.close()


def test_batch_full_size_sampled():
    """The 256-segment ragged batch (lengths log-uniform in [2^10, 2^24],
    seed 4, targets over the eight nu and exp->normal), checked on samples."""
    lens, targets = W.ragged_segments(4, 256)
    spec, ins, outs = make_batch(lens, targets)
    b = qm.Batch(spec)
    b.run()
    torch.cuda.synchronize()
    rng = np.random.default_rng(1)
    for j in range(0, 256, 3):
        x, o = ins[j], outs[j]
        idx = torch.from_numpy(rng.integers(0, x.numel(), min(512, x.numel()))).to(DEV)
        w = oracle_of(spec[j], x[idx].cpu().numpy())
        assert not f64_violations(o[idx].cpu().numpy(), w, 1e-12).any(), j
        assert not torch.isnan(o).any()
    b.close()
    del ins, outs
    torch.cuda.empty_cache()


def test_batch_uniform_segments_match_the_streaming_kernel_bit_for_bit():
    """Uniform -> normal segments of the batch evaluate the same fixed-point
    table as the streaming FP64 kernel, with the offset t_u turned into a
    double by integer normalisation instead of the exact FP64 add; both are
    exact, so the results must be identical.  The inputs crowd the top
    segment next to u = 1/2, where the offset and the inner 32-bit chain
    pass through 0, plus the tail-stress mixture."""
    rng = np.random.default_rng(41)
    k = np.concatenate([2**52 + rng.integers(-2**46, 2**46, 1 << 18), 2**52 + np.arange(-4096, 4096)])
    near = k.astype(np.float64) * 2.0**-53
    mix = W.mixture_f64(43, 1 << 18).numpy()
    u = torch.from_numpy(np.concatenate([near, mix])).to(DEV)
    zb = torch.empty_like(u)
    zs = torch.empty_like(u)
    zf = torch.empty_like(u)
    b = qm.Batch([(qm.QM_DIST_UNIFORM, qm.QM_DIST_NORMAL, 0.0, u, zb)])
    b.run()
    torch.cuda.synchronize()
    b.close()
    b = qm.Batch([(qm.QM_DIST_UNIFORM, qm.QM_DIST_NORMAL, 0.0, u, zs)])
    b.run_separate()
    torch.cuda.synchronize()
    b.close()
    qm.qm_normal_quantile_f64(u, zf, qm.QM_VAR_FIXED)
    torch.cuda.synchronize()
    assert torch.equal(zb, zf) and torch.equal(zs, zf)
