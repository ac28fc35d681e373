#!/usr/bin/env python3
"""Benchmark of the quantile hot path on GB300.

Workload (one step): the FP64 normal quantile z = Phi^{-1}(u) over n = 2^28
doubles resident in HBM -- the seed-2 tail-stress mixture (90 % k 2^-53
uniforms, 10 % 2^-e m with e up to 990, mirrored with probability 1/2) --
through the library's default FP64 path (qm_normal_quantile_f64).  Inputs and
outputs (2 GiB each) are far larger than L2, so no flush is needed.

Prints ONE JSON line (rank 0).  Under torchrun each rank processes its own
2^28-element slice of the same counter-based stream (weak scaling, no
collective on the data path).  --impl reference times the CPU FP64 oracle on a
bounded sample of the same workload instead.
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
NOMINAL_FP64_TFLOPS = 1.25     # GB300 nominal dense FP64 (profiling recipe table)


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--n-log2", type=int, default=28, help="elements per rank = 2^n")
    p.add_argument("--variant", default="default")
    p.add_argument("--no-extras", action="store_true", help="skip variant/e2e/cpu legs")
    return p.parse_args()


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


def run_reference(args, rank, world):
    if rank != 0:
        return
    import oracle
    from paper_0901_0638_gb300 import workloads as W
    threads = oracle.threads_used(0)
    m = 1 << 20  # bounded per-step sample of the workload
    u = W.mixture_f64(2, m).numpy()
    for _ in range(args.warmup):
        oracle.probit(u[: 1 << 14])
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.probit(u)
        times.append(time.perf_counter() - t0)
    t = sum(times) / len(times)
    val = m / t / 1e9
    line = {"metric": METRIC, "value": val, "unit": "Gsamples/s", "n_gpus": 0, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": "fp64 normal quantile, seed-2 tail-stress mixture, per-step sample 2^20 of 2^28",
                       "n": 1 << 28, "sample": m},
            "cpu_baseline": {"value": val, "unit": "Gsamples/s", "cores": threads, "kind": "oracle",
                             "sample": f"2^20 elements of the 2^28 workload per step"},
            "e2e": {"value": val, "unit": "Gsamples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)

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
    variants = {"default": qm.QM_VAR_DEFAULT, "table": qm.QM_VAR_TABLE, "compact": qm.QM_VAR_COMPACT,
                "branchfree": qm.QM_VAR_BRANCHFREE, "hybrid_vote": qm.QM_VAR_HYBRID_VOTE,
                "mixed_halley": qm.QM_VAR_MIXED_HALLEY, "cuda_normcdfinv": qm.QM_VAR_CUDA_LIBM}
    var = variants[args.variant]
    u = W.mixture_f64(2, n, first=rank * n, device=dev)
    z = torch.empty_like(u)
    stream = torch.cuda.current_stream(dev)
    # algorithmic DP work: table path for d >= 2^-65, deep rational below
    d = torch.minimum(u, 1.0 - u)
    n_deep = int(((d > 0) & (d < 2.0 ** -65)).sum())
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
    ms = ev0.elapsed_time(ev1) / args.steps
    if pg is not None:
        t = torch.tensor([ms], device=dev)
        pg.all_reduce(t, op=pg.ReduceOp.MAX)
        ms = float(t.item())
    value = world * n / (ms * 1e-3) / 1e9

    # roofline of the dominant kernel (FP64 table kernel): FP64-issue bound.
    # Algorithmic FP64 work per element: table path 7 FMA + 1 add = 15 flops;
    # deep-tail rational ~ 26 FMA (Horner) + 7 (reciprocal) + log ~ 2 x 45 flops.
    flops = (n - n_deep - n_edge) * 15 + n_deep * 90
    achieved = flops / (ms * 1e-3) / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": NOMINAL_FP64_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / NOMINAL_FP64_TFLOPS, "traffic": None,
                "peak_source": "nominal GB300 FP64 1.25 TFLOP/s (recipe table); measured DFMA issue 1.20 TFLOP/s",
                "hbm_view": {"achieved_gbs": 16 * n / (ms * 1e-3) / 1e9, "peak_gbs": 6780.7,
                             "frac": 16 * n / (ms * 1e-3) / 1e9 / 6780.7}}

    extras = {}
    cpu = None
    e2e = None
    if not args.no_extras and rank == 0:
        # other FP64 variants on the same inputs (context)
        ev_a = torch.cuda.Event(enable_timing=True)
        ev_b = torch.cuda.Event(enable_timing=True)
        for name, v in variants.items():
            if name == args.variant:
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
        # FP32 normal quantile on the 24-bit Philox grid at the same n (HBM bound)
        del z
        _, u32 = W.uniform24(1, n, device=dev)
        z32 = torch.empty_like(u32)
        for name, v in (("table", qm.QM_VAR_TABLE), ("sqrt_form", qm.QM_VAR_SQRT_FORM),
                        ("paper_form", qm.QM_VAR_BRANCHFREE), ("cuda_normcdfinvf", qm.QM_VAR_CUDA_LIBM)):
            qm.qm_normal_quantile_f32(u32, z32, v, stream=stream)
            torch.cuda.synchronize(dev)
            ev_a.record(stream)
            for _ in range(5):
                qm.qm_normal_quantile_f32(u32, z32, v, stream=stream)
            ev_b.record(stream)
            torch.cuda.synchronize(dev)
            t = ev_a.elapsed_time(ev_b) / 5
            extras[f"fp32_{name}"] = {"ms": t, "gsamples_s": n / (t * 1e-3) / 1e9,
                                      "hbm_frac": 8 * n / (t * 1e-3) / 1e9 / 6780.7}
        del u32, z32
        z = torch.empty_like(u)
        # end to end through the C ABI with host buffers (pinned), copies timed
        hu = u.cpu().pin_memory()
        hz = torch.empty_like(hu).pin_memory()
        for _ in range(2):
            u.copy_(hu, non_blocking=True)
            qm.qm_normal_quantile_f64(u, z, var, stream=stream)
            hz.copy_(z, non_blocking=True)
        torch.cuda.synchronize(dev)
        ev_a.record(stream)
        k2 = max(1, min(args.steps, 5))
        for _ in range(k2):
            u.copy_(hu, non_blocking=True)
            qm.qm_normal_quantile_f64(u, z, var, stream=stream)
            hz.copy_(z, non_blocking=True)
        ev_b.record(stream)
        torch.cuda.synchronize(dev)
        t = ev_a.elapsed_time(ev_b) / k2
        e2e = {"value": n / (t * 1e-3) / 1e9, "unit": "Gsamples/s",
               "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": 8 * n, "ms_per_step": t,
               "note": "pinned host -> device copy, kernel, device -> host copy, one stream"}
        del hu, hz
        cpu = cpu_oracle_leg(n)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "Gsamples/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic",
                "config": {"workload": "fp64 normal quantile Phi^-1, n=2^28 doubles per GPU, seed-2 "
                                       "tail-stress mixture (90% k*2^-53, 10% 2^-e*m mirrored)",
                           "n_per_gpu": n, "variant": args.variant, "l2": "inputs larger than L2 (4 GiB)",
                           "deep_tail_elements": n_deep, "edge_elements": n_edge},
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": args.steps, "clocks": clocks, "variants": extras}
        print(json.dumps(line), flush=True)
    if pg is not None:
        pg.barrier()
        pg.destroy_process_group()


if __name__ == "__main__":
    main()
