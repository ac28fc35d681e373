"""The continuous-batching server: every request's samples are the same
alone and in the mix, match the oracle, memory admission holds, and the
plain (one launch per request) baseline serves the same trace."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
import paper_0901_0638_gb300 as qm
from paper_0901_0638_gb300 import workloads as W
from tests.gpu_util import d2h, f32_violations, f64_violations

pytestmark = pytest.mark.gpu


def small_trace(count=240, seed=5, rate=2e4, lo=8, hi=15):
    tr = W.serving_trace(seed, rate=rate, seconds=1.0, lo=lo, hi=hi, max_requests=count)
    for r in tr:
        r["id"] = r["key"]
    return tr


def fetch(c):
    torch.cuda.synchronize()
    return d2h(c.out, c.n, np.float64 if c.is_f64 else np.float32)


def expected(c, m=None):
    """Oracle values of the first m samples of a completed request."""
    n = c.n if m is None else min(m, c.n)
    if c.kind == qm.QM_REQ_NORMAL_F32:
        k = oracle.philox_stream(c.key, 0, n) >> 8
        return oracle.probit((k.astype(np.float64) + 0.5) * 2.0**-24), None
    words = oracle.philox_stream(c.key, 0, 2 * n).astype(np.uint64)
    kk = ((words[0::2] >> 11) << 32) | words[1::2]
    upper = kk >= 2**52
    d = (np.where(upper, 2**53 - 1 - kk, kk).astype(np.float64) + 0.5) * 2.0**-53
    if c.kind == qm.QM_REQ_EXP_NORMAL:
        x = np.where(upper, -np.log1p(-d), -np.log(d))
        return oracle.recycle_exp(x), x
    z = oracle.probit(d)
    z = np.where(upper, -z, z)
    if c.kind == qm.QM_REQ_STUDENT_T:
        return oracle.recycle_t(c.nu, z), None
    return z, None


def check_parity(c, got, m=4096):
    w, x = expected(c, m)
    g = got[: len(w)]
    if c.kind == qm.QM_REQ_NORMAL_F32:
        assert not f32_violations(g, w).any()
    elif c.kind == qm.QM_REQ_EXP_NORMAL:
        slope = np.exp(-x) / (np.exp(-0.5 * w * w) / np.sqrt(2 * np.pi))
        assert np.all(np.abs(g - w) <= 1e-12 * np.abs(w) + 4 * 2.2e-16 * x * slope)
    elif c.kind == qm.QM_REQ_STUDENT_T:
        assert not f64_violations(g, w, 1e-12).any()
    else:
        assert not f64_violations(g, w, 4e-15).any()


def test_batched_results_equal_alone_and_match_oracle():
    trace = small_trace()
    srv = qm.Server(mem_budget=1 << 30, max_batch=64, streams=2)
    done = srv.replay(trace)
    assert len(done) == len(trace) and all(c.status == 0 for c in done)
    assert srv.stats()["launches"] < len(trace)              # requests were batched
    mixed = {c.id: (c, fetch(c)) for c in done}
    alone_srv = qm.Server(mem_budget=1 << 30, max_batch=1, streams=1)
    kinds = set()
    for r in trace[:60]:
        (c_alone,) = alone_srv.replay([dict(r, t_arrival=0.0)])
        a = fetch(c_alone)
        c, m = mixed[r["id"]]
        assert np.array_equal(a, m), r                         # bit-identical
        check_parity(c, m)
        kinds.add(c.kind)
        alone_srv.release(c_alone.id)
    assert kinds == {0, 1, 2, 3}
    for c in done:
        srv.release(c.id)
    srv.close()
    alone_srv.close()


def test_student_t_requests_with_untabulated_nu():
    """Requests with any real nu in range (run-time tables, built at submit)."""
    srv = qm.Server(mem_budget=1 << 28, max_batch=16, streams=2)
    trace = [{"id": i, "n": 3000 + 17 * i, "kind": qm.QM_REQ_STUDENT_T, "nu": nu, "key": 700 + i,
              "t_arrival": 0.0} for i, nu in enumerate([2.7, 0.9, 4.0, 55.0, 2.7])]
    done = srv.replay(trace)
    assert len(done) == len(trace) and all(c.status == 0 for c in done)
    for c in done:
        check_parity(c, fetch(c))
        srv.release(c.id)
    srv.close()


def test_memory_admission_bounds_in_flight_bytes():
    budget = 4 << 20
    trace = [{"id": i, "n": 1 << 17, "kind": qm.QM_REQ_NORMAL_F64, "key": 100 + i, "t_arrival": 0.0}
             for i in range(24)]                                # 1 MiB each, 24 MiB total
    srv = qm.Server(mem_budget=budget, max_batch=64, streams=2, release_on_done=True)
    done = srv.replay(trace)
    assert len(done) == 24
    # at most four outputs fit at once, so at least six launches were needed
    assert srv.stats()["launches"] >= 6
    admits = sorted((c.t_admit, c.t_done) for c in done)
    for t_admit, _ in admits:
        live = sum(1 for a, d in admits if a <= t_admit < d)
        assert live <= 4
    srv.close()


def test_plain_baseline_serves_the_same_trace():
    trace = small_trace(count=120, seed=6)
    plain = qm.Server(mem_budget=1 << 30, max_batch=1, streams=1, release_on_done=False)
    batched = qm.Server(mem_budget=1 << 30, max_batch=64, streams=2, release_on_done=False)
    a = {c.id: fetch(c) for c in plain.replay(trace)}
    b = {c.id: fetch(c) for c in batched.replay(trace)}
    assert a.keys() == b.keys()
    assert all(np.array_equal(a[k], b[k]) for k in a)
    assert plain.stats()["launches"] == len(trace)
    plain.close()
    batched.close()


def test_server_argument_errors():
    srv = qm.Server(mem_budget=1 << 20, max_batch=8, streams=1)
    with pytest.raises(qm.QMError) as e:
        srv.submit({"n": 16, "kind": 9, "key": 1})
    assert e.value.status == qm.QM_ERR_INVALID
    with pytest.raises(qm.QMError) as e:
        srv.submit({"n": 16, "kind": qm.QM_REQ_STUDENT_T, "nu": 0.5, "key": 1})
    assert e.value.status == qm.QM_ERR_UNSUPPORTED
    with pytest.raises(qm.QMError) as e:
        srv.submit({"n": 1 << 20, "kind": qm.QM_REQ_NORMAL_F64, "key": 1})   # 8 MiB > 1 MiB
    assert e.value.status == qm.QM_ERR_NOMEM
    srv.close()


def test_replay_timeout_returns_status_and_server_keeps_serving():
    """Failure detection on the host: a replay whose bounded wait runs out
    returns QM_ERR_TIMEOUT at its limit (the wait is a host loop, nothing on
    the GPU is left waiting), and the same server then serves a new trace
    with correct results."""
    import time
    srv = qm.Server(mem_budget=1 << 26, max_batch=16, streams=2)
    # request 1 arrives at once; request 2 only after the replay's 0.05 s limit
    trace = [{"id": 1, "n": 4096, "kind": qm.QM_REQ_NORMAL_F64, "key": 901, "t_arrival": 0.0},
             {"id": 2, "n": 4096, "kind": qm.QM_REQ_NORMAL_F64, "key": 902, "t_arrival": 5.0}]
    t0 = time.perf_counter()
    with pytest.raises(qm.QMError) as e:
        srv.replay(trace, timeout_s=0.05)
    assert e.value.status == qm.QM_ERR_TIMEOUT
    assert time.perf_counter() - t0 < 2.0          # gave up at its limit, not at request 2
    assert "of 2 done" in qm.qm_last_error()
    time.sleep(0.2)
    stale = srv.poll()                             # request 1 may complete after the timeout
    assert all(c.id == 1 and c.status == 0 for c in stale)
    srv.release(1)
    # the same server serves a fresh trace: every kind, oracle parity
    trace2 = [{"id": 10 + k, "n": 3000 + 97 * k, "kind": kind, "nu": 4.0, "key": 910 + k,
               "t_arrival": 0.001 * k} for k, kind in enumerate(range(4))]
    done = srv.replay(trace2, timeout_s=60.0)
    assert sorted(c.id for c in done) == [10, 11, 12, 13] and all(c.status == 0 for c in done)
    for c in done:
        check_parity(c, fetch(c))
        srv.release(c.id)
    srv.close()
