#!/usr/bin/env python3
"""Benchmark of the quantile hot path on GB300.

Workload (one step): the FP64 normal quantile z = Phi^{-1}(u) over n = 2^28
doubles resident in HBM -- the seed-2 tail-stress mixture (90 % k 2^-53
uniforms, 10 % 2^-e m with e up to 990, mirrored with probability 1/2) --
through the library's default FP64 path (qm_normal_quantile_f64, the
fixed-point segment kernel k_f64_fixed).  Inputs and
outputs (2 GiB each) are far larger than L2, so no flush is needed.

Prints ONE JSON line (rank 0).  Under torchrun each rank processes its own
2^28-element slice of the same counter-based stream (weak scaling, no
collective on the data path).  --impl reference times the CPU FP64 oracle on a
bounded sample of the same workload instead.

Beside the headline, the default run (rank 0) adds: the other FP64 and FP32
variants on the same inputs, the end-to-end figure on pinned host buffers,
the CPU oracle on a bounded sample, and three legs with their own clock
records -- "fused" (Philox -> FP32 Phi^{-1} for 2^32 samples, written and as
moments, the moments asserted within 5 sigma of 0, 1, 0, 3), "batch" (the
256-segment ragged recycling batch, one graph launch against one launch per
segment) and "serving" (the Poisson request trace, continuous batching
against one plain launch per request, with p50/p99 latency).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Φ^{-1} Gsamples/s FP32/FP64 & % roofline; batched p50/p99 latency vs plain"
FP64_WORKLOAD = ("fp64 normal quantile Phi^-1, n=2^28 doubles per GPU, seed-2 tail-stress mixture "
                 "(90% k*2^-53, 10% 2^-e*m mirrored)")
NOMINAL_FP64_TFLOPS = 1.25     # GB300 nominal dense FP64 (profiling recipe table)
SMS, SCHEDULERS, LANES, MAX_SM_GHZ = 152, 4, 32, 2.07
ISSUE_PEAK_TINSTR = SMS * SCHEDULERS * LANES * MAX_SM_GHZ / 1e3   # thread-instructions/ns -> T/s
# Issue rates measured on this GPU by probe kernels (thread-level operations
# per second, 2.07 GHz): FP64 FMA 0.50-0.60 T/s, FP32 FMA 36-37 T/s, MUFU
# 4.8 T/s.  They price the method's arithmetic in the composite roofline.
DFMA_PER_S, FFMA_PER_S, MUFU_PER_S = 0.55e12, 36.5e12, 4.8e12
FALLBACK_HBM_GBS = 6800.0      # profiling recipe fallback, used only without the measured file
# ncu counters (DRAM bytes and issued instructions per element) are recorded
# in profiles/counters.json together with a fingerprint of the kernel's
# sources; a counter whose kernel has changed since is not used (traffic null).
COUNTERS_JSON = os.path.join(ROOT, "profiles", "counters.json")
KERNEL_FILES = {
    "k_f64_fixed": ["paper_0901_0638_gb300/csrc/qm_fixed.cu", "paper_0901_0638_gb300/csrc/qm_fx.cuh",
                    "paper_0901_0638_gb300/csrc/qm_fx_tables.h", "paper_0901_0638_gb300/_build.py"],
    "k_f32_table": ["paper_0901_0638_gb300/csrc/qm_quantile.cu", "paper_0901_0638_gb300/csrc/qm_device.cuh",
                    "paper_0901_0638_gb300/csrc/qm_tables.h", "paper_0901_0638_gb300/_build.py"],
}


def hbm_peak():
    """Measured HBM copy bandwidth (GB/s) and where it came from."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            v = float(json.load(f)["hbm_gbs"])
        return v, "measured (MEASURED_PEAKS.json hbm_gbs, STREAM-style copy)"
    except (OSError, KeyError, ValueError):
        return FALLBACK_HBM_GBS, "fallback 6.8 TB/s (no measured peak file)"


def kernel_fingerprint(kernel):
    """Hash of the kernel's sources with comments and whitespace removed."""
    import hashlib
    import re
    h = hashlib.sha256()
    for rel in KERNEL_FILES[kernel]:
        with open(os.path.join(ROOT, rel)) as f:
            src = f.read()
        if rel.endswith(".py"):
            src = re.sub(r"#[^\n]*", "", src)
        else:
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            src = re.sub(r"//[^\n]*", "", src)
        h.update(re.sub(r"\s+", " ", src).encode())
    return h.hexdigest()[:16]


def recorded_counters(kernel):
    """The ncu counters of `kernel` if they were taken on its current sources."""
    try:
        with open(COUNTERS_JSON) as f:
            rec = json.load(f).get(kernel)
    except (OSError, ValueError):
        return None
    if not rec or rec.get("fingerprint") != kernel_fingerprint(kernel):
        return None
    return rec


def record_counters(csv_path, n, command):
    """Reads an ncu --csv --print-units base metrics log (details page) and
    stores, per kernel of KERNEL_FILES found in it, DRAM bytes and issued
    instructions per element (averaged over its launches, n elements each)."""
    import csv
    import re
    rows = {}
    with open(csv_path) as f:
        lines = [ln for ln in f if ln.startswith('"')]
    for r in csv.DictReader(lines):
        name = r.get("Kernel Name", "")
        k = next((k for k in KERNEL_FILES if re.search(r"\b" + k + r"\b", name)), None)
        if k is None:
            continue
        launch = rows.setdefault(k, {}).setdefault(r["ID"], {})
        launch[r["Metric Name"]] = float(r["Metric Value"].replace(",", ""))
    try:
        with open(COUNTERS_JSON) as f:
            out = json.load(f)
    except (OSError, ValueError):
        out = {}
    for k, launches in rows.items():
        ls = list(launches.values())
        avg = lambda m: sum(x.get(m, 0.0) for x in ls) / len(ls)
        out[k] = {"fingerprint": kernel_fingerprint(k), "n": n, "launches": len(ls),
                  "dram_bytes_per_element": (avg("dram__bytes_read.sum") + avg("dram__bytes_write.sum")) / n,
                  "inst_per_element": 32 * avg("smsp__inst_executed.sum") / n,
                  "duration_ns": avg("gpu__time_duration.sum"), "command": command,
                  "per_launch": {m: avg(m) for m in sorted(ls[0])}}
    with open(COUNTERS_JSON, "w") as f:
        json.dump(out, f, indent=1, sort_keys=True)
        f.write("\n")
    print(json.dumps(out, indent=1))


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n-log2", type=int, default=28, help="elements per rank = 2^n")
    p.add_argument("--variant", default="default")
    p.add_argument("--no-extras", action="store_true", help="skip variant/e2e/cpu legs")
    p.add_argument("--cpu-threads", type=int, default=0,
                   help="host threads of the oracle in --impl reference (0: all cores)")
    p.add_argument("--workload", default="fp64", choices=["fp64", "fp32", "batch", "serve", "fused",
                                                          "hyperbolic", "copula", "tcopula"],
                   help="fp64: the headline line; fp32/batch/serve: the other hot-path kernels "
                        "(for profiling and context)")
    p.add_argument("--serve-seconds", type=float, default=10.0,
                   help="length of the serving trace (the serving leg and --workload serve)")
    p.add_argument("--no-legs", action="store_true",
                   help="default run: skip the fused, batch and serving legs")
    p.add_argument("--record-counters", metavar="NCU_CSV", default=None,
                   help="store per-element DRAM bytes and instructions of the kernels in an ncu "
                        "--csv --print-units base log (n = 2^--n-log2 per launch) in profiles/, "
                        "then exit (no GPU needed)")
    p.add_argument("--counters-command", default="", help="the command that produced NCU_CSV")
    p.add_argument("--batch-hi", type=int, default=24,
                   help="ragged batch: segment lengths log-uniform in [2^10, 2^hi]")
    return p.parse_args()


def shard_first(rank: int, n_per_rank: int) -> int:
    """First element of rank's slice of the counter-based input stream."""
    return rank * n_per_rank


def max_over_ranks(ms: float, pg, device=None) -> float:
    """The slowest rank's step time (weak scaling: value = world n / max)."""
    if pg is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except FileNotFoundError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        loaded = [s for s in sm if mx and s > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def cpu_oracle_leg(n_total: int, budget_s: float = 12.0):
    """The CPU FP64 oracle, as it stands, on a bounded prefix of the same
    workload (same generator), all host cores."""
    import oracle
    from paper_0901_0638_gb300 import workloads as W
    threads = oracle.threads_used(0)
    probe = W.mixture_f64(2, 1 << 14).numpy()
    t0 = time.perf_counter()
    oracle.probit(probe)
    per = (time.perf_counter() - t0) / probe.size
    m = int(min(n_total, max(1 << 16, budget_s / max(per, 1e-9))))
    u = W.mixture_f64(2, m).numpy()
    t0 = time.perf_counter()
    oracle.probit(u)
    dt = time.perf_counter() - t0
    return {"value": m / dt / 1e9, "unit": "Gsamples/s", "cores": threads, "kind": "oracle",
            "sample": f"first {m} elements of the seed-2 mixture (of 2^28), {dt:.1f} s"}


T2_VOTE_D_MIN = 1.0373472162855378e-3   # d above this <=> t_2 coordinate below 15.5 (Sec. 7.3)


def vote_t2_fraction(u):
    """Share of the warp votes of the HYBRID_VOTE kernel that take the t_2
    rational: the kernel votes over aligned groups of 32 consecutive
    elements, and a group takes t_2 only if every d = min(u, 1 - u) lies in
    its domain (lanes past the end count as inside).  A property of the input
    and of the kernel's grouping, computed from the input."""
    import torch
    d = torch.minimum(u, 1.0 - u)
    ok = d > T2_VOTE_D_MIN
    pad = (-ok.numel()) % 32
    if pad:
        ok = torch.cat([ok, torch.ones(pad, dtype=torch.bool, device=ok.device)])
    return float(ok.view(-1, 32).all(dim=1).float().mean())


def reference_sample(args, nt):
    """The oracle's work for one step of the reference arm: a bounded sample
    of the workload `args.workload`, from the same generators as the device
    path.  Returns (fn, elements per call, config, dtype)."""
    import numpy as np
    import oracle
    from paper_0901_0638_gb300 import workloads as W
    if args.workload == "fp64":
        m = 1 << 20
        u = W.mixture_f64(2, m).numpy()
        cfg = {"workload": FP64_WORKLOAD, "n_per_gpu": 1 << 28,
               "sample": "each step evaluates the first 2^20 of the 2^28 elements", "sample_n": m}
        return (lambda: oracle.probit(u, nt)), m, cfg, "f64"
    if args.workload == "fp32":
        n = 1 << args.n_log2
        m = min(n, 1 << 20)
        _, u32 = W.uniform24(1, m)
        u = u32.double().numpy()
        cfg = {"workload": f"fp32 normal quantile, n=2^{args.n_log2} floats, u=fl32((k+1/2)2^-24), "
                           "k = top 24 bits of Philox seed 1",
               "sample": f"each step evaluates the first {m} of the {n} elements in FP64", "sample_n": m}
        return (lambda: oracle.probit(u, nt)), m, cfg, "f64"
    if args.workload == "batch":
        lens, targets = W.ragged_segments(4, 256, hi=args.batch_hi)
        segs = []
        for j, (nj, tg) in enumerate(zip(lens, targets)):
            mj = min(int(nj), 4096)
            if tg == 8:
                segs.append((None, W.exponential(4, mj, 0, j + 1).numpy()))
            else:
                segs.append((W.NU_SET[tg], W.normal_box_muller(4, mj, 0, j + 1).numpy()))
        m = sum(x.size for _, x in segs)

        def fn():
            for nu, x in segs:
                if nu is None:
                    oracle.recycle_exp(x, nt)
                else:
                    oracle.recycle_t(nu, x, nt)
        cfg = {"workload": "ragged recycling batch: 256 segments, lengths log-uniform [2^10, 2^24] "
                           "(seed 4), normal->t_nu for nu in {1,2,3,4,5,8,10,30} and exp->normal",
               "sample": "stratified: the first min(len, 4096) elements of every segment", "sample_n": m}
        return fn, m, cfg, "f64"
    if args.workload == "fused":
        chunks, w = 256, 4096

        def fn():
            for c in range(chunks):
                k = oracle.philox_stream(3, c << 24, w) >> 8
                oracle.probit((k.astype(np.float64) + 0.5) * 2.0 ** -24, nt)
        cfg = {"workload": "fused Philox4x32-10 (seed 3) -> fp32 normal, n=2^32",
               "sample": "256 chunks of 4096 samples at stride 2^24 (2^20 of the 2^32), Philox and "
                         "quantile both in the oracle", "sample_n": chunks * w}
        return fn, chunks * w, cfg, "f64"
    return None, 0, None, None


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    nt = max(0, args.cpu_threads)
    threads = oracle.threads_used(nt)
    fn, m, cfg, dtype = reference_sample(args, nt)
    if fn is None:
        print(json.dumps({"impl": "reference", "unavailable": f"no CPU oracle leg for the "
                          f"{args.workload} workload (its parity is checked in tests/)"}), flush=True)
        return
    for _ in range(args.warmup):
        fn()
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        fn()
        times.append(time.perf_counter() - t0)
    t = sum(times) / len(times)
    val = m / t / 1e9
    line = {"metric": METRIC, "value": val, "unit": "Gsamples/s", "n_gpus": args.gpus, "device": "cpu (host cores)",
            "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": dtype, "data": "synthetic", "impl": "reference",
            "config": cfg,
            "cpu_baseline": {"value": val, "unit": "Gsamples/s", "cores": threads, "kind": "oracle",
                             "sample": cfg["sample"]},
            "e2e": {"value": val, "unit": "Gsamples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def timed(fn, stream, steps, warmup):
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(steps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps


# 5-sigma bounds of the first four sample moments of 2^32 standard normals:
# sd(z^k) = sqrt(1, 2, 15, 96) (E z^2 = 1, Var z^2 = 2, E z^6 = 15,
# Var z^4 = 105 - 9) over sqrt(2^32)
MOMENT_5SIGMA_2P32 = (7.6e-5, 1.1e-4, 3.0e-4, 7.5e-4)


def fused_leg(qm, dev, stream, n_log2=32, steps=3, warmup=1, gpu_index=0):
    """Fused Philox4x32-10 (seed 3) -> FP32 Phi^{-1} for 2^n_log2 samples,
    written (4 B each) and, separately, reduced on the device to the first
    four moments, which must lie within 5 sigma of (0, 1, 0, 3) at 2^32;
    then the FP64 sampler (53-bit grid) for 2^(n_log2 - 2) samples written."""
    import torch
    n = 1 << n_log2
    out = torch.empty(n, dtype=torch.float32, device=dev)
    mom = torch.empty(4, dtype=torch.float64, device=dev)
    clk = ClockSampler(gpu_index)
    clk.start()
    ms_w = timed(lambda: qm.qm_sample_fused(qm.QM_DIST_NORMAL, 3, 0, out, stream=stream),
                 stream, steps, warmup)
    ms_m = timed(lambda: qm.qm_sample_fused(qm.QM_DIST_NORMAL, 3, 0, None, n=n, moments4=mom,
                                            stream=stream), stream, steps, warmup)
    clocks = clk.stop()
    m = (mom / n).cpu().tolist()
    del out
    dev_m = [abs(m[0]), abs(m[1] - 1.0), abs(m[2]), abs(m[3] - 3.0)]
    bounds = [b * (2.0 ** 16 / 2.0 ** (n_log2 / 2)) for b in MOMENT_5SIGMA_2P32]
    assert all(x < b for x, b in zip(dev_m, bounds)), f"fused moments {m} outside 5 sigma {bounds}"
    n64 = n >> 2
    out64 = torch.empty(n64, dtype=torch.float64, device=dev)
    ms_64 = timed(lambda: qm.qm_sample_fused(qm.QM_DIST_NORMAL, 3, 0, out64, out_is_f64=True,
                                             stream=stream), stream, steps, warmup)
    del out64
    peak, _ = hbm_peak()
    return {"workload": f"fused Philox4x32-10 (seed 3) -> fp32 Phi^-1, n=2^{n_log2}: written "
                        f"({4 * n >> 30} GiB) and moments only; fp64 sampler 2^{n_log2 - 2} written",
            "n": n, "written": {"ms": ms_w, "gsamples_s": n / (ms_w * 1e-3) / 1e9,
                                "write_gbs": 4 * n / (ms_w * 1e-3) / 1e9,
                                "hbm_frac_of_write": 4 * n / (ms_w * 1e-3) / 1e9 / peak},
            "moments": {"ms": ms_m, "gsamples_s": n / (ms_m * 1e-3) / 1e9, "mean": m[0], "m2": m[1],
                        "m3": m[2], "m4": m[3], "check": "within 5 sigma of (0, 1, 0, 3)",
                        "bounds": bounds, "passed": True},
            "fp64_written": {"n": n64, "ms": ms_64, "gsamples_s": n64 / (ms_64 * 1e-3) / 1e9,
                             "hbm_frac_of_write": 8 * n64 / (ms_64 * 1e-3) / 1e9 / peak},
            "bound": "alu (Philox integer work; no HBM traffic for uniforms)", "clocks": clocks}


def batch_leg(qm, W, dev, stream, hi=24, steps=10, warmup=3, tune=True, gpu_index=0):
    """256 ragged recycling segments (seed 4, lengths log-uniform in
    [2^10, 2^hi]): one persistent graph launch against one plain launch per
    segment, after the autotuner has picked the tiles."""
    import torch
    lens, targets = W.ragged_segments(4, 256, hi=hi)
    spec = []
    for j, (nj, tg) in enumerate(zip(lens, targets)):
        if tg == 8:
            x = W.exponential(4, nj, 0, j + 1, dev)
            spec.append((qm.QM_DIST_EXPONENTIAL, qm.QM_DIST_NORMAL, 0.0, x, torch.empty_like(x)))
        else:
            x = W.normal_box_muller(4, nj, 0, j + 1, dev)
            spec.append((qm.QM_DIST_NORMAL, qm.QM_DIST_STUDENT_T, W.NU_SET[tg], x, torch.empty_like(x)))
    b = qm.Batch(spec)
    if tune:
        b.tune(reps=3, stream=stream)
    tuning = b.tuning()
    tot = int(sum(lens))
    clk = ClockSampler(gpu_index)
    clk.start()
    ms = timed(lambda: b.run(stream), stream, steps, warmup)
    ms_sep = timed(lambda: b.run_separate(stream), stream, steps, warmup)
    clocks = clk.stop()
    b.close()
    del spec
    return {"workload": f"ragged recycling batch: 256 segments, lengths log-uniform [2^10, 2^{hi}] "
                        "(seed 4), normal->t_nu for nu in {1,2,3,4,5,8,10,30} and exp->normal",
            "elements": tot, "tuning": tuning, "autotuned": tune,
            "graph": {"ms": ms, "gsamples_s": tot / (ms * 1e-3) / 1e9, "launches": 1},
            "separate_launches": {"ms": ms_sep, "gsamples_s": tot / (ms_sep * 1e-3) / 1e9,
                                  "launches": sum(1 for x in lens if x)},
            "speedup": ms_sep / ms, "clocks": clocks}


def serving_leg(qm, W, seconds=10.0, gpu_index=0):
    """The serving trace (Poisson 2e4 requests/s, seed 5, n log-uniform in
    [2^8, 2^24], four target kinds, 8 GiB admission budget), replayed in
    real time through continuous batching and through one plain launch per
    request (FIFO, one stream): sustained Gsamples/s, p50/p99 latency."""
    import numpy as np
    tr = W.serving_trace(5, rate=2e4, seconds=seconds)
    for r in tr:
        r["id"] = r["key"]
    tot = sum(r["n"] for r in tr)
    res = {}
    clk = ClockSampler(gpu_index)
    clk.start()
    for name, mb, st in (("batched", 512, 2), ("plain", 1, 1)):
        srv = qm.Server(mem_budget=8 << 30, max_batch=mb, streams=st, release_on_done=True)
        done = srv.replay(tr, timeout_s=900)
        lat = np.array([c.t_done - c.t_arrival for c in done])
        span = max(c.t_done for c in done) - min(c.t_arrival for c in done)
        res[name] = {"gsamples_s": tot / span / 1e9, "p50_ms": 1e3 * float(np.percentile(lat, 50)),
                     "p99_ms": 1e3 * float(np.percentile(lat, 99)), "makespan_s": span,
                     "launches": srv.stats()["launches"]}
        srv.close()
    res["clocks"] = clk.stop()
    res.update({"workload": f"serving: Poisson 2e4 req/s for {seconds} s (seed 5), n log-uniform "
                            "[2^8, 2^24], 4 target kinds, 8 GiB budget",
                "requests": len(tr), "samples": tot, "offered_gsamples_s": tot / seconds / 1e9})
    return res


def side_workload(args):
    """fp32 / fused / batch / serve / hyperbolic / copula workloads: one JSON
    line each (rank 0 only)."""
    import torch
    import paper_0901_0638_gb300 as qm
    from paper_0901_0638_gb300 import workloads as W
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    qm.load()
    peak, peak_src = hbm_peak()
    line = {"metric": METRIC, "unit": "Gsamples/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "data": "synthetic"}
    if args.workload == "fp32":
        n = 1 << args.n_log2
        _, u = W.uniform24(1, n, device=dev)
        z = torch.empty_like(u)
        ms = timed(lambda: qm.qm_normal_quantile_f32(u, z, qm.QM_VAR_DEFAULT, stream=stream),
                   stream, args.steps, args.warmup)
        gbs = 8 * n / (ms * 1e-3) / 1e9
        rec = recorded_counters("k_f32_table")
        line.update(value=n / (ms * 1e-3) / 1e9, ms_per_step=ms, dtype="f32",
                    config={"workload": f"fp32 normal quantile, n=2^{args.n_log2} floats, "
                                        "u=fl32((k+1/2)2^-24), k = top 24 bits of Philox seed 1"},
                    roofline={"bound": "hbm", "kernel": "k_f32_table", "achieved": gbs, "peak": peak,
                              "unit": "GB/s", "frac": gbs / peak, "peak_source": peak_src,
                              "traffic": rec["dram_bytes_per_element"] * n if rec else None,
                              "algorithmic_bytes_per_element": 8})
    elif args.workload == "fused":
        n_log2 = args.n_log2 if args.n_log2 != 28 else 32
        r = fused_leg(qm, dev, stream, n_log2, args.steps, args.warmup)
        line.update(value=r["written"]["gsamples_s"], ms_per_step=r["written"]["ms"], dtype="f32",
                    config={"workload": r["workload"], "n": r["n"]}, fused=r)
    elif args.workload == "hyperbolic":
        # exponential -> hyperbolic recycling (alpha, beta, delta) = (1.3, 0.4, 0.7)
        # over 2^n two-sided exponential base samples resident in HBM
        n = 1 << args.n_log2
        a, b, d = 1.3, 0.4, 0.7
        g = torch.Generator(device=dev)
        g.manual_seed(6)
        e = torch.empty(n, dtype=torch.float64, device=dev).exponential_(generator=g)
        side = torch.rand(n, dtype=torch.float64, device=dev, generator=g) < 0.5
        v = torch.where(side, e / (a - b), -e / (a + b))
        del e, side
        x = torch.empty_like(v)
        h = qm.Hyperbolic(a, b, d)
        ms = timed(lambda: h.recycle(v, x, stream=stream), stream, args.steps, args.warmup)
        line.update(value=n / (ms * 1e-3) / 1e9, ms_per_step=ms, dtype="f64",
                    config={"workload": f"exponential -> hyperbolic recycling (alpha, beta, delta) = "
                                        f"({a}, {b}, {d}), n=2^{args.n_log2} two-sided exponential samples"},
                    roofline={"bound": "alu", "note": "biased fixed-point segment rows (integer "
                                                      "chain, one exact FP64 add and one DFMA per "
                                                      "element); 16 B/element",
                              "hbm_frac": 16 * n / (ms * 1e-3) / 1e9 / peak})
        h.close()
    elif args.workload in ("copula", "tcopula"):
        # Gaussian copula (or t copula with nu = 4), d = 8, equicorrelation
        # 0.5, margins alternating normal / Student t (nu = 4, 2.7 run-time
        # table, 30), 2^n samples
        import numpy as np
        n = 1 << (args.n_log2 if args.n_log2 != 28 else 24)
        d = 8
        R = np.full((d, d), 0.5) + 0.5 * np.eye(d)
        L = np.linalg.cholesky(R)
        margins = [(qm.QM_DIST_NORMAL, 0.0), (qm.QM_DIST_STUDENT_T, 4.0), (qm.QM_DIST_NORMAL, 0.0),
                   (qm.QM_DIST_STUDENT_T, 2.7)] * 2
        margins[-1] = (qm.QM_DIST_STUDENT_T, 30.0)
        tnu = 4.0 if args.workload == "tcopula" else None
        c = qm.Copula(L, margins, nu=tnu)
        out = torch.empty(d * n, dtype=torch.float64, device=dev)
        ms = timed(lambda: c.sample(11, 0, out, n, stream=stream), stream, args.steps, args.warmup)
        line.update(value=n / (ms * 1e-3) / 1e9, unit="Gsamples/s (d-dimensional)", ms_per_step=ms,
                    dtype="f64",
                    config={"workload": ("t copula nu=4" if tnu else "Gaussian copula") +
                                        f" d={d}, equicorrelation 0.5, normal/t margins, "
                                        f"n=2^{n.bit_length() - 1} samples, Philox4x32-10 in registers",
                            "values_per_s": d * n / (ms * 1e-3)},
                    roofline={"bound": "alu", "note": "FP64: d normals (fixed point, 1 DFMA each) + "
                                                      "d(d+1)/2 FMA + t maps per sample; 8 d B written "
                                                      "per sample",
                              "hbm_frac_of_write": 8 * d * n / (ms * 1e-3) / 1e9 / peak})
        c.close()
    elif args.workload == "batch":
        r = batch_leg(qm, W, dev, stream, args.batch_hi, args.steps, args.warmup)
        line.update(value=r["graph"]["gsamples_s"], ms_per_step=r["graph"]["ms"], dtype="f64",
                    config={"workload": r["workload"], "elements": r["elements"]}, batch=r)
    else:
        r = serving_leg(qm, W, args.serve_seconds)
        line.update(value=r["batched"]["gsamples_s"], ms_per_step=None, dtype="mixed",
                    config={"workload": r["workload"], "requests": r["requests"], "samples": r["samples"],
                            "offered_gsamples_s": r["offered_gsamples_s"]}, serving=r)
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.record_counters:
        return record_counters(args.record_counters, 1 << args.n_log2, args.counters_command)
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.workload != "fp64":
        if rank == 0:
            side_workload(args)
        return

    import torch
    import paper_0901_0638_gb300 as qm
    from paper_0901_0638_gb300 import workloads as W

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        pg = dist

    def barrier():
        if pg is not None:
            pg.barrier()

    qm.load()
    n = 1 << args.n_log2
    variants = {"default": qm.QM_VAR_DEFAULT, "fixed": qm.QM_VAR_FIXED, "table": qm.QM_VAR_TABLE,
                "compact": qm.QM_VAR_COMPACT,
                "branchfree": qm.QM_VAR_BRANCHFREE, "hybrid_vote": qm.QM_VAR_HYBRID_VOTE,
                "mixed_halley": qm.QM_VAR_MIXED_HALLEY, "almost_normal": qm.QM_VAR_ALMOST_NORMAL,
                "t2_multi": qm.QM_VAR_T2_MULTI, "paper_exact": qm.QM_VAR_PAPER_EXACT,
                "paper_exact_b": qm.QM_VAR_PAPER_EXACT_B, "cuda_normcdfinv": qm.QM_VAR_CUDA_LIBM}
    var = variants[args.variant]
    u = W.mixture_f64(2, n, first=shard_first(rank, n), device=dev)
    z = torch.empty_like(u)
    stream = torch.cuda.current_stream(dev)
    # input classes of the mixture (context for the line)
    d = torch.minimum(u, 1.0 - u)
    n_deep = int(((d > 0) & (d < 2.0 ** -65)).sum())
    n_sub = int(((d > 0) & (d < 2.0 ** -1022)).sum())
    n_edge = int((d <= 0).sum())
    del d

    def step():
        qm.qm_normal_quantile_f64(u, z, var, stream=stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize(dev)
    barrier()
    sampler = ClockSampler(local)
    sampler.start()
    torch.cuda.synchronize(dev)
    barrier()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        step()
    ev1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    clocks = sampler.stop()
    ms = max_over_ranks(ev0.elapsed_time(ev1) / args.steps, pg, dev)
    value = world * n / (ms * 1e-3) / 1e9

    # roofline of the dominant kernel, on the method's algorithmic work per
    # element: the slower of its bytes at the measured HBM copy bandwidth and
    # its arithmetic at the measured issue rates (FIXED: 16 B, one FP64 FMA,
    # and the six multiply-adds of its degree-6 segment polynomial, which the
    # kernel runs on the integer pipes, priced at the FP32 FMA rate; the
    # branchy FP64 variants: about 45-60 FP64 operations).
    secs = ms * 1e-3
    peak, peak_src = hbm_peak()
    gbs = 16 * n / secs / 1e9
    fixed = args.variant in ("default", "fixed")
    fp64_ops = 1 if fixed else 50
    terms = {"hbm_ps": 16 / (peak * 1e9) * 1e12, "fp64_ps": fp64_ops / DFMA_PER_S * 1e12,
             "fp32_ps": (6 if fixed else 0) / FFMA_PER_S * 1e12}
    bound = max(terms, key=terms.get)
    t_elem = secs / n
    rec = recorded_counters("k_f64_fixed") if fixed else None
    roofline = {"bound": "hbm" if bound == "hbm_ps" else "alu",
                "kernel": "k_f64_fixed" if fixed else args.variant,
                "achieved": gbs if bound == "hbm_ps" else fp64_ops * n / secs / 1e12,
                "peak": peak if bound == "hbm_ps" else DFMA_PER_S / 1e12,
                "unit": "GB/s" if bound == "hbm_ps" else "T FP64 FMA/s",
                "frac": terms[bound] * 1e-12 / t_elem,
                "peak_source": peak_src if bound == "hbm_ps" else "measured FP64 FMA issue rate (probe)",
                "traffic": rec["dram_bytes_per_element"] * n if rec else None,
                "algorithmic_bytes_per_element": 16,
                "terms_ps_per_element": terms, "measured_ps_per_element": t_elem * 1e12,
                "hbm_frac_of_nominal_7900": gbs / 7900.0}
    if rec:
        # implementation efficiency, not the roofline: the kernel's own issued
        # instructions (ncu, on these sources) against the issue-slot peak
        roofline["issue_view"] = {"inst_per_element": rec["inst_per_element"],
                                  "achieved_tinstr_s": rec["inst_per_element"] * n / secs / 1e12,
                                  "peak_tinstr_s": ISSUE_PEAK_TINSTR,
                                  "frac": rec["inst_per_element"] * n / secs / 1e12 / ISSUE_PEAK_TINSTR,
                                  "counters": "profiles/counters.json (" + rec["command"] + ")"}

    extras = {}
    legs = {}
    cpu = None
    e2e = None
    if not args.no_extras and rank == 0:
        # other FP64 variants on the same inputs (context)
        ev_a = torch.cuda.Event(enable_timing=True)
        ev_b = torch.cuda.Event(enable_timing=True)
        for name, v in variants.items():
            if name == args.variant or (name == "fixed" and args.variant == "default"):
                continue
            qm.qm_normal_quantile_f64(u, z, v, stream=stream)
            torch.cuda.synchronize(dev)
            ev_a.record(stream)
            reps = 3
            for _ in range(reps):
                qm.qm_normal_quantile_f64(u, z, v, stream=stream)
            ev_b.record(stream)
            torch.cuda.synchronize(dev)
            t = ev_a.elapsed_time(ev_b) / reps
            extras[f"fp64_{name}"] = {"ms": t, "gsamples_s": n / (t * 1e-3) / 1e9}
            if name in ("hybrid_vote", "paper_exact"):
                extras[f"fp64_{name}"]["votes_taking_t2"] = vote_t2_fraction(u)
        # the branchy variants on 53-bit uniforms alone (seed 8, no tail
        # stress): the inputs where the vote and the extra t_2 branch matter
        del z
        uu = W.uniform53(8, n, device=dev)
        zu = torch.empty_like(uu)
        uni = {}
        for name in ("fixed", "compact", "hybrid_vote", "t2_multi", "almost_normal", "paper_exact",
                     "paper_exact_b"):
            v = variants[name]
            qm.qm_normal_quantile_f64(uu, zu, v, stream=stream)
            torch.cuda.synchronize(dev)
            ev_a.record(stream)
            for _ in range(3):
                qm.qm_normal_quantile_f64(uu, zu, v, stream=stream)
            ev_b.record(stream)
            torch.cuda.synchronize(dev)
            t = ev_a.elapsed_time(ev_b) / 3
            uni[name] = {"ms": t, "gsamples_s": n / (t * 1e-3) / 1e9}
            if name in ("hybrid_vote", "paper_exact"):
                uni[name]["votes_taking_t2"] = vote_t2_fraction(uu)
        extras["fp64_uniform53_only"] = uni
        del uu, zu
        z = torch.empty_like(u)
        # FP32 normal quantile on the 24-bit Philox grid at the same n (HBM bound)
        del z
        _, u32 = W.uniform24(1, n, device=dev)
        z32 = torch.empty_like(u32)
        for name, v in (("table", qm.QM_VAR_TABLE), ("sqrt_form", qm.QM_VAR_SQRT_FORM),
                        ("paper_form", qm.QM_VAR_BRANCHFREE), ("paper_exact", qm.QM_VAR_PAPER_EXACT),
                        ("almost_normal", qm.QM_VAR_ALMOST_NORMAL),
                        ("cuda_normcdfinvf", qm.QM_VAR_CUDA_LIBM)):
            qm.qm_normal_quantile_f32(u32, z32, v, stream=stream)
            torch.cuda.synchronize(dev)
            ev_a.record(stream)
            for _ in range(5):
                qm.qm_normal_quantile_f32(u32, z32, v, stream=stream)
            ev_b.record(stream)
            torch.cuda.synchronize(dev)
            t = ev_a.elapsed_time(ev_b) / 5
            extras[f"fp32_{name}"] = {"ms": t, "gsamples_s": n / (t * 1e-3) / 1e9,
                                      "hbm_frac": 8 * n / (t * 1e-3) / 1e9 / peak}
        del u32, z32
        z = torch.empty_like(u)
        # end to end through the C ABI with host buffers (pinned): the kernel
        # reads u from and writes z to page-locked host memory over the host
        # link (unified addressing: the pinned pointer is a device pointer), so
        # every step moves its 2^28 inputs host -> device and its 2^28 results
        # device -> host inside the timed region, in one launch.  Beside it, a
        # copy-engine pipeline (2^24-element chunks over four streams: copy
        # in, kernel, copy out) on the same buffers.
        hu = u.cpu().pin_memory()
        hz = torch.empty_like(hu).pin_memory()

        def e2e_step():
            qm.qm_normal_quantile_f64(hu, hz, var, stream=stream)

        chunk = min(n, 1 << 24)
        streams = [torch.cuda.Stream(dev) for _ in range(4)]

        def pipe_step():
            cur = torch.cuda.current_stream(dev)
            for st in streams:
                st.wait_stream(cur)
            for i, c0 in enumerate(range(0, n, chunk)):
                st = streams[i % len(streams)]
                with torch.cuda.stream(st):
                    sl = slice(c0, min(n, c0 + chunk))
                    u[sl].copy_(hu[sl], non_blocking=True)
                    qm.qm_normal_quantile_f64(u[sl], z[sl], var, stream=st)
                    hz[sl].copy_(z[sl], non_blocking=True)
            for st in streams:
                cur.wait_stream(st)

        def time_host(step):
            for _ in range(2):
                step()
            torch.cuda.synchronize(dev)
            ev_a.record(stream)
            k2 = max(1, min(args.steps, 5))
            for _ in range(k2):
                step()
            ev_b.record(stream)
            torch.cuda.synchronize(dev)
            return ev_a.elapsed_time(ev_b) / k2

        # the host link's own copy rate on the same buffers: copy engines
        # moving the 2^28 inputs host -> device and 2^28 results device ->
        # host at the same time (two streams); no library call
        def link_step():
            cur = torch.cuda.current_stream(dev)
            for st in streams[:2]:
                st.wait_stream(cur)
            with torch.cuda.stream(streams[0]):
                u.copy_(hu, non_blocking=True)
            with torch.cuda.stream(streams[1]):
                hz.copy_(z, non_blocking=True)
            for st in streams[:2]:
                cur.wait_stream(st)

        t_pipe = time_host(pipe_step)
        t_link = time_host(link_step)
        hz.zero_()
        t = time_host(e2e_step)
        idx = torch.arange(0, n, 4099)
        qm.qm_normal_quantile_f64(u, z, var, stream=stream)
        torch.cuda.synchronize(dev)
        assert torch.equal(hz[idx], z[idx.to(dev)].cpu())
        e2e = {"value": n / (t * 1e-3) / 1e9, "unit": "Gsamples/s",
               "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * n, "ms_per_step": t,
               "note": "pinned host buffers passed to qm_normal_quantile_f64: the kernel streams u from "
                       "and z to host memory over the host link (zero-copy), one launch per step",
               "gpu_launches_per_step": 1,
               "copy_engine_pipeline": {"ms_per_step": t_pipe, "value": n / (t_pipe * 1e-3) / 1e9,
                                        "note": "2^24-element chunks over four streams: copy in, "
                                                "kernel, copy out"},
               "link_roofline": {"bound": "host link", "unit": "GB/s",
                                 "achieved": 16 * n / (t * 1e-3) / 1e9,
                                 "peak": 16 * n / (t_link * 1e-3) / 1e9,
                                 "frac": t_link / t,
                                 "peak_source": "measured in this run: copy engines moving the step's "
                                                "inputs in and results out concurrently on the same "
                                                "pinned buffers"}}
        del hu, hz
        cpu = cpu_oracle_leg(n)
        if not args.no_legs:
            # the other configurations of the metric, each with its own clocks:
            # fused generate+transform at 2^32 (moments asserted within 5
            # sigma), the ragged batch (graph vs one launch per segment), and
            # the serving trace (continuous batching vs one launch per request)
            del u, z
            torch.cuda.empty_cache()
            legs["fused"] = fused_leg(qm, dev, stream, gpu_index=local)
            torch.cuda.empty_cache()
            legs["batch"] = batch_leg(qm, W, dev, stream, gpu_index=local)
            torch.cuda.empty_cache()
            legs["serving"] = serving_leg(qm, W, args.serve_seconds, gpu_index=local)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "Gsamples/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic",
                "config": {"workload": FP64_WORKLOAD,
                           "n_per_gpu": n, "variant": args.variant, "l2": "inputs larger than L2 (4 GiB)",
                           "deep_tail_elements": n_deep, "subnormal_d_elements": n_sub,
                           "edge_elements": n_edge,
                           "dominant_kernel": "k_f64_fixed" if args.variant in ("default", "fixed")
                                              else args.variant},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": args.steps, "clocks": clocks, "variants": extras, **legs}
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.barrier()
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
