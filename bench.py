#!/usr/bin/env python
"""Benchmark: |M|^2 events/s for g g -> t tbar g g on GB300 (mixed vs FP64).

One step = the whole hot path over one batch: seeded RAMBO phase space with
gluon cuts on the device (rambo_sample) + helicity- and colour-summed |M|^2
(me_sigmakin) for 2^20 events at sqrt(s) = 1.5 TeV.  The momenta batch
(201 MB) is larger than L2, so no flush is needed between steps.

  python bench.py [--gpus N --steps K --warmup W]           # this library
  python bench.py --impl reference [...]                    # FP64 CPU oracle

Multi-GPU (torchrun, one rank per GPU): every rank evaluates its own event
range (weak scaling, no data-path collective); the timed region is bracketed by
barriers and the maximum over ranks is reported.  Prints one JSON line.
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
sys.path.insert(0, ROOT)

METRIC = "|M|^2 events/s gg->t tbar gg (mixed vs FP64, 1 GB300); serving p50/p99 latency"
# dominant kernel of the mixed-precision step, per workload
KERNELS = {"ee_mumu": "me_kernel_scalar<ee_mumu, float>", "gg_ttx": "me_kernel_scalar<gg_ttx, float>",
           "gg_ttxg": "me_kernel_tab<gg_ttxg, float>", "gg_ttxgg": "me_kernel_tab<gg_ttxgg, float>",
           "gg_ttxggg": "me_kernel_interp<gg_ttxggg, float>",
           "uux_epem": "me_kernel_scalar<uux_epem, float>", "uux_epemg": "me_kernel_scalar<uux_epemg, float>",
           "uux_epemgg": "me_kernel_tab<uux_epemgg, float>", "uux_epemggg": "me_kernel_tab<uux_epemggg, float>"}
PROCESS_LABEL = {"ee_mumu": "e+ e- -> mu+ mu-", "gg_ttx": "g g -> t t~", "gg_ttxg": "g g -> t t~ g",
                 "gg_ttxgg": "g g -> t t~ g g", "gg_ttxggg": "g g -> t t~ g g g",
                 "uux_epem": "u u~ -> e+ e-", "uux_epemg": "u u~ -> e+ e- g", "uux_epemgg": "u u~ -> e+ e- g g",
                 "uux_epemggg": "u u~ -> e+ e- g g g"}
DY_NGLUON = {"uux_epem": 0, "uux_epemg": 1, "uux_epemgg": 2, "uux_epemggg": 3}


def oracle_me2(name, mom):
    """The FP64 CPU oracle's |M|^2 for a workload (QCD / e+e- or Drell-Yan)."""
    import oracle
    from paper_2507_21039_gb300.workloads import ALPHA_S, MT, workload

    if name in DY_NGLUON:
        return oracle.dy_me2(DY_NGLUON[name], mom, alpha_s=ALPHA_S)
    return oracle.me2(name, mom, mt=MT, alpha=workload(name).alpha)
FP32_LANES_PER_SM = 128     # FP32 FMA lanes per SM (4 SMSPs x 32)


def n_sm() -> int:
    """SM count of the current device (152 on GB300), queried, not assumed."""
    import torch

    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--workload", default="gg_ttxgg")
    ap.add_argument("--fp64-steps", type=int, default=2)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the gg -> t t~ ggg configuration added to the headline line")
    ap.add_argument("--serving-requests", type=int, default=500,
                    help="requests per load point of the serving sweep (the definition's 2000 take ~8 minutes)")
    ap.add_argument("--small", action="store_true",
                    help="the small processes (ee -> mu mu, gg -> t t~): HBM GB/s, launch overhead, FP-pipe fraction")
    ap.add_argument("--case", nargs=3, metavar=("WORKLOAD", "PRECISION", "NEVT"),
                    help="profiling case: sample NEVT events, then one warm and one measured me_sigmakin")
    return ap.parse_args()


# ------------------------------------------------------------------ helpers
class ClockSampler:
    """nvidia-smi sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.file = None

    def __enter__(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or self.file is None:
            return None
        self.file.flush()
        rows = []
        with open(self.file.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.file.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup(want_cuda=True):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist

        backend = "nccl" if (want_cuda and torch.cuda.is_available()) else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist

        dist.barrier()


def allreduce_max(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def cpu_baseline(name, seconds, rank):
    """The FP64 CPU oracle as it stands, on the host cores, on a bounded sample."""
    import oracle
    from paper_2507_21039_gb300.workloads import DR_MIN, PT_MIN, workload

    w = workload(name)
    mom, _, _ = oracle.rambo(w.seed, w.sqrt_s, w.masses_final, 0, 256, w.cut_mask, PT_MIN, DR_MIN)
    t = time.perf_counter()
    oracle_me2(name, mom)
    rate = 256 / (time.perf_counter() - t)
    n = int(max(256, min(1 << 17, rate * seconds)))
    mom, _, _ = oracle.rambo(w.seed, w.sqrt_s, w.masses_final, 0, n, w.cut_mask, PT_MIN, DR_MIN)
    t = time.perf_counter()
    oracle_me2(name, mom)
    dt = time.perf_counter() - t
    # one core, on a sample of about a sixth of the time
    cores = oracle.max_threads()
    n1 = int(max(64, min(n, (n / dt) / cores * seconds / 6)))
    out = {"value": n / dt, "unit": "events/s", "cores": cores, "kind": "oracle",
           "sample": f"first {n} events of the {name} workload (seed {w.seed}), FP64 Berends-Giele "
                     f"colour-ordered recursion + brute-force colour matrix, all helicities, "
                     f"OpenMP over events; {dt:.1f} s"}
    if name not in DY_NGLUON:  # the oracle's Drell-Yan entry point has no thread limit
        from paper_2507_21039_gb300.workloads import MT

        t = time.perf_counter()
        oracle.me2(name, mom[:n1], mt=MT, alpha=w.alpha, nthreads=1)
        dt1 = time.perf_counter() - t
        out["single_core"] = {"value": n1 / dt1, "unit": "events/s", "cores": 1,
                              "sample": f"first {n1} events, one thread; {dt1:.1f} s"}
    return out


# ------------------------------------------------------------------ arms
def run_reference(args):
    world, rank, _ = dist_setup(want_cuda=False)
    if rank != 0:
        return
    import oracle
    from paper_2507_21039_gb300.workloads import DR_MIN, PT_MIN, workload

    name = args.workload
    w = workload(name)
    oracle.build()
    # size each step so that warmup + steps end within a few minutes
    mom, _, _ = oracle.rambo(w.seed, w.sqrt_s, w.masses_final, 0, 128, w.cut_mask, PT_MIN, DR_MIN)
    t = time.perf_counter()
    oracle_me2(name, mom)
    rate = 128 / (time.perf_counter() - t)
    per_step = max(64, int(rate * min(20.0, 150.0 / max(1, args.steps + args.warmup))))
    times = []
    for s in range(args.warmup + args.steps):
        mom, _, _ = oracle.rambo(w.seed, w.sqrt_s, w.masses_final, s * per_step, per_step, w.cut_mask, PT_MIN, DR_MIN)
        t = time.perf_counter()
        oracle_me2(name, mom)
        dt = time.perf_counter() - t
        if s >= args.warmup:
            times.append(dt)
    total = sum(times)
    value = per_step * len(times) / total
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "events/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": name, "events_per_step": per_step, "sqrt_s": w.sqrt_s, "seed": w.seed,
                   "precision": "fp64", "note": "reference arm = FP64 CPU oracle (the paper ships no code)"},
        "cpu_baseline": {"value": value, "unit": "events/s", "cores": oracle.max_threads(), "kind": "oracle",
                         "sample": f"{per_step} events per step of the {name} workload"},
        "e2e": {"value": value, "unit": "events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def run_ours(args):
    import torch

    world, rank, local = dist_setup(want_cuda=True)
    import __graft_entry__

    __graft_entry__.build()
    import paper_2507_21039_gb300 as me
    from paper_2507_21039_gb300.workloads import workload

    torch.cuda.set_device(local)
    name = args.workload
    w = workload(name)
    n = w.nevt
    masses = [0.0, 0.0] + list(w.masses_final)
    cuts = me.cuts_for(name)
    ev0 = rank * n  # weak scaling: each rank owns its own event range
    stream = torch.cuda.current_stream()
    mom = torch.empty((n, w.npar, 4), dtype=torch.float64, device="cuda")
    me2 = torch.empty(n, dtype=torch.float64, device="cuda")
    h_mixed = me.workload_handle(name, "mixed")
    h_fp64 = me.workload_handle(name, "fp64")
    me.rambo_sample(w.seed, ev0, n, w.sqrt_s, masses, cuts, momenta_out=mom, check=True)
    me.me_filter_helicities(h_mixed, mom)
    me.me_filter_helicities(h_fp64, mom)
    ngood = len(me.me_good_helicities(h_mixed))

    def step(h, seed_ev0, ev_pair=None):
        me.rambo_sample(w.seed, seed_ev0, n, w.sqrt_s, masses, cuts, momenta_out=mom, stream=stream)
        if ev_pair:
            ev_pair[0].record(stream)
        me.me_sigmakin(h, mom, me2, stream=stream)
        if ev_pair:
            ev_pair[1].record(stream)

    def timed(h, steps, warmup, clocks=False):
        for s in range(warmup):
            step(h, ev0)
        torch.cuda.synchronize()
        barrier(world)
        torch.cuda.synchronize()
        s0 = torch.cuda.Event(enable_timing=True)
        s1 = torch.cuda.Event(enable_timing=True)
        kern = []
        sampler = ClockSampler(local) if clocks else None
        if sampler:
            sampler.__enter__()
        pairs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        s0.record(stream)
        for s in range(steps):
            step(h, ev0, pairs[s])
        s1.record(stream)
        torch.cuda.synchronize()
        kern = [a.elapsed_time(b) for a, b in pairs]
        if sampler:
            sampler.__exit__(None, None, None)
        barrier(world)
        elapsed = s0.elapsed_time(s1) / 1e3
        return elapsed, kern, (sampler.summary() if sampler else None)

    elapsed, kern_ms, clocks = timed(h_mixed, args.steps, args.warmup, clocks=(rank == 0))
    elapsed_max = allreduce_max(elapsed, world)
    value = n * world * args.steps / elapsed_max
    me_ms = statistics.mean(kern_ms)

    el64, kern64, _ = timed(h_fp64, args.fp64_steps, 1)
    el64 = allreduce_max(el64, world)
    value64 = n * world * args.fp64_steps / el64

    # end to end through the C ABI with host buffers (pinned), the same step:
    # rambo_sample into host momenta (D2H), me_sigmakin from host momenta (H2D)
    # into host |M|^2 (D2H); every copy inside the timed region
    host_mom = torch.empty((n, w.npar, 4), dtype=torch.float64, pin_memory=True)
    host_me2 = torch.empty(n, dtype=torch.float64, pin_memory=True)

    def host_step():
        me.rambo_sample(w.seed, ev0, n, w.sqrt_s, masses, cuts, momenta_out=host_mom)
        me.me_sigmakin(h_mixed, host_mom, host_me2)

    host_step()
    barrier(world)
    t = time.perf_counter()
    for _ in range(args.e2e_steps):
        host_step()
    e2e_dt = allreduce_max(time.perf_counter() - t, world)
    e2e = {"value": n * world * args.e2e_steps / e2e_dt, "unit": "events/s",
           "h2d_bytes_per_step": host_mom.numel() * 8,
           "d2h_bytes_per_step": host_mom.numel() * 8 + host_me2.numel() * 8,
           "path": "rambo_sample into pinned host momenta, me_sigmakin from them into pinned host |M|^2"}

    chain_f, colour_f = me.me_flops_per_event(h_mixed)
    flops = (chain_f + colour_f) * n
    peaks, peak_src = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    nsm = n_sm()
    fp32_peak = nsm * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12
    achieved = flops / (me_ms / 1e3) / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                "frac": achieved / fp32_peak, "traffic": None,
                "kernel": KERNELS[name],
                "peak_source": f"derived: {nsm} SMs (queried) x {FP32_LANES_PER_SM} FP32 lanes x 2 flops x "
                               f"{sm_max:.0f} MHz ({peak_src} sm_max_mhz)",
                "flops_per_event": chain_f + colour_f, "me_kernel_ms": me_ms}
    # DRAM bytes of one launch from the committed ncu summary, if it was taken on
    # this kernel version (same generator flop count); null otherwise
    slug = KERNELS[name].replace("<", "_").replace(">", "").replace(", float", "_f32").replace(" ", "")
    traffic_file = os.path.join(ROOT, "profiles", f"{slug}.traffic.txt")
    if os.path.exists(traffic_file):
        kv = {}
        with open(traffic_file) as f:
            for line in f:
                if "=" in line and not line.startswith("#"):
                    k, v = line.strip().split("=", 1)
                    kv[k] = v
        if kv.get("kernel") == roofline["kernel"] and float(kv.get("flops_per_event", -1)) == roofline["flops_per_event"]:
            roofline["traffic"] = float(kv["bytes_per_event"]) * n

    out = {
        "metric": METRIC, "value": value, "unit": "events/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * elapsed_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": name, "process": PROCESS_LABEL[name], "global_batch": n * world,
                   "events_per_gpu": n, "sqrt_s": w.sqrt_s, "seed": w.seed, "precision": "mixed",
                   "cuts": "gluon pT > 20 GeV, pairwise dR > 0.4", "good_helicities": ngood,
                   "l2": (f"inputs larger than L2 (momenta {n * w.npar * 32 / 1e6:.0f} MB per step)"
                          if n * w.npar * 32 > 129e6 else
                          f"momenta {n * w.npar * 32 / 1e6:.0f} MB per step, smaller than L2; no flush "
                          "(the kernel is bound by arithmetic, not memory)"),
                   "step": "rambo_sample (device) + me_sigmakin", "parallelism": f"replicas x{world}"},
        "fp64": {"value": value64, "unit": "events/s", "ms_per_step": 1e3 * el64 / args.fp64_steps,
                 "me_kernel_ms": statistics.mean(kern64)},
        "mixed_over_fp64": value / value64,
        "e2e": e2e,
        "gpu_launches": 2 * args.steps,
        "roofline": roofline,
        "clocks": clocks,
    }
    if name == "gg_ttxgg" and world == 1 and not args.no_extra:
        out["gg_ttxggg"] = extra_workload(me, "gg_ttxggg", steps=3, warmup=2, fp64_steps=1)
    if not args.no_serving and rank == 0:
        from paper_2507_21039_gb300 import serving

        sw = serving.sweep(nreq=args.serving_requests)
        point = next(p for p in sw["points"] if p["load"] == 0.7)
        out["serving"] = dict(point, requests=sw["requests_per_point"], mean_batch=sw["mean_batch"],
                              saturation_events_per_s=sw["saturation_events_per_s"], processes=sw["processes"],
                              precision=sw["precision"], lanes=sw["lanes"])
        out["serving_sweep"] = sw
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(name, args.cpu_seconds, rank)
    if rank == 0:
        print(json.dumps(out), flush=True)
    h_mixed.close()
    h_fp64.close()
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()


def extra_workload(me, name, steps, warmup, fp64_steps):
    """Another benchmark configuration on this GPU, reported beside the
    headline: the same step (device RAMBO + |M|^2 on the workload's batch),
    mixed and FP64, CUDA events on the launching stream, and the mixed
    kernel's fraction of the derived FP32 peak."""
    import torch

    from paper_2507_21039_gb300.workloads import workload

    w = workload(name)
    n = w.nevt
    masses = [0.0, 0.0] + list(w.masses_final)
    cuts = me.cuts_for(name)
    stream = torch.cuda.current_stream()
    mom = torch.empty((n, w.npar, 4), dtype=torch.float64, device="cuda")
    me2 = torch.empty(n, dtype=torch.float64, device="cuda")
    me.rambo_sample(w.seed, 0, n, w.sqrt_s, masses, cuts, momenta_out=mom, check=True)
    res = {"workload": name, "process": PROCESS_LABEL[name], "events_per_step": n, "sqrt_s": w.sqrt_s,
           "seed": w.seed, "step": "rambo_sample (device) + me_sigmakin"}
    for prec, st, wu in (("mixed", steps, warmup), ("fp64", fp64_steps, 0)):
        h = me.workload_handle(name, prec)
        me.me_filter_helicities(h, mom)
        for _ in range(wu):
            me.rambo_sample(w.seed, 0, n, w.sqrt_s, masses, cuts, momenta_out=mom, stream=stream)
            me.me_sigmakin(h, mom, me2, stream=stream)
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(st)]
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        for a, b in ev:
            me.rambo_sample(w.seed, 0, n, w.sqrt_s, masses, cuts, momenta_out=mom, stream=stream)
            a.record(stream)
            me.me_sigmakin(h, mom, me2, stream=stream)
            b.record(stream)
        s1.record(stream)
        torch.cuda.synchronize()
        dt = s0.elapsed_time(s1) / 1e3
        kms = statistics.mean(a.elapsed_time(b) for a, b in ev)
        res[prec] = {"value": n * st / dt, "unit": "events/s", "steps": st, "warmup": wu,
                     "ms_per_step": 1e3 * dt / st, "me_kernel_ms": kms}
        if prec == "mixed":
            chain_f, colour_f = me.me_flops_per_event(h)
            peaks, peak_src = measured_peaks()
            fp32_peak = n_sm() * FP32_LANES_PER_SM * 2 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
            achieved = (chain_f + colour_f) * n / (kms / 1e3) / 1e12
            res["roofline"] = {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                               "frac": achieved / fp32_peak, "kernel": KERNELS[name],
                               "flops_per_event": chain_f + colour_f, "peak_source": f"derived ({peak_src})"}
        h.close()
    res["mixed_over_fp64"] = res["mixed"]["value"] / res["fp64"]["value"]
    return res


def run_small():
    """ee -> mu mu and gg -> t t~ at their workload sizes: |M|^2 kernel time
    (CUDA events, momenta resident), HBM GB/s of the algorithmic bytes
    (32 npar + 8 per event), FP32-pipe fraction of the generator flops, and the
    launch overhead (host time of a one-event me_sigmakin call against its
    device time)."""
    import torch

    import paper_2507_21039_gb300 as me
    from paper_2507_21039_gb300.workloads import WORKLOADS

    peaks, _ = measured_peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = n_sm() * FP32_LANES_PER_SM * 2 * sm_max * 1e6
    out = {}
    for name in ("ee_mumu", "gg_ttx"):
        w = WORKLOADS[name]
        masses = [0.0, 0.0] + list(w.masses_final)
        mom = me.rambo_sample(w.seed, 0, w.nevt, w.sqrt_s, masses, me.cuts_for(name), check=True)
        for prec in ("fp64", "fp32"):
            h = me.workload_handle(name, prec)
            me.me_filter_helicities(h, mom)
            me2 = me.me_sigmakin(h, mom)
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            s0.record()
            for _ in range(20):
                me.me_sigmakin(h, mom, me2)
            s1.record()
            torch.cuda.synchronize()
            t = s0.elapsed_time(s1) / 20 / 1e3
            chain_f, colour_f = me.me_flops_per_event(h)
            one, one_out = mom[:1].clone(), me2[:1].clone()
            for _ in range(50):
                me.me_sigmakin(h, one, one_out)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(1000):
                me.me_sigmakin(h, one, one_out)
            torch.cuda.synchronize()
            host = (time.perf_counter() - t0) / 1000
            s0.record()
            for _ in range(1000):
                me.me_sigmakin(h, one, one_out)
            s1.record()
            torch.cuda.synchronize()
            dev = s0.elapsed_time(s1) / 1000 / 1e3
            h.close()
            out[f"{name}/{prec}"] = {
                "events": w.nevt, "kernel_ms": t * 1e3, "events_per_s": w.nevt / t,
                "hbm_gb_s": w.nevt * (32 * w.npar + 8) / t / 1e9,
                "fp32_pipe_fraction": (chain_f + colour_f) * w.nevt / t / fp32_peak,
                "one_event_call_us": {"host": host * 1e6, "device": dev * 1e6}}
    print(json.dumps(out))


def run_case(name, prec, nevt):
    """Small fixed case for ncu captures: sampler, filter, two |M|^2 launches."""
    import torch

    import __graft_entry__

    __graft_entry__.build()
    import paper_2507_21039_gb300 as me
    from paper_2507_21039_gb300.workloads import workload

    w = workload(name)
    masses = [0.0, 0.0] + list(w.masses_final)
    mom = me.rambo_sample(w.seed, 0, nevt, w.sqrt_s, masses, me.cuts_for(name), check=True)
    h = me.workload_handle(name, prec)
    me.me_filter_helicities(h, mom[:4096])
    out = me.me_sigmakin(h, mom)
    torch.cuda.synchronize()
    out = me.me_sigmakin(h, mom)
    torch.cuda.synchronize()
    print(json.dumps({"case": name, "precision": prec, "nevt": nevt, "checksum": float(out.sum())}))
    h.close()


if __name__ == "__main__":
    a = parse()
    if a.case:
        run_case(a.case[0], a.case[1], int(a.case[2]))
    elif a.small:
        run_small()
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
