"""Benchmark of the GB300 hybrid Quicksort (one JSON line on stdout).

Headline workload: qs_sort_f64 on n = 2^28 FP64 keys uniform in [-1e6, 1e6]
(seeded, synthetic).  One step = one in-place sort of one such array through
the C-ABI: the persistent partition kernel (pivot selection, partition passes
with decoupled look-back, recursion) plus the Bitonic leaf kernel.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Timing: every step sorts its own pristine copy of the input (2 GiB, larger
than L2), so the K timed steps run back to back with no restore inside the
timed region; device time comes from CUDA events on the launching stream,
bracketed by a barrier and torch.cuda.synchronize().  With N > 1 (torchrun)
each rank sorts its own array (replicas, weak scaling); the time is the max
over ranks and the value counts the keys of all ranks.

--impl reference times the CPU oracle (single thread) on a bounded sample of
the same workload; it is the baseline arm, not a GPU implementation.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import re
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

LOG2N = 28
N_KEYS = 1 << LOG2N
WORKLOAD = "f64 sort, n=2^%d, uniform [-1e6,1e6] (seed 0x5EED0002), in place"
HBM_FALLBACK_GBS = 6800.0


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return HBM_FALLBACK_GBS, "fallback"


def _kernel_source_sha1() -> str:
    """SHA-1 of the kernel sources with their // comments, trailing blanks and
    empty lines removed, so that a change of comments alone keeps the DRAM
    traffic recorded from an ncu capture (the sources hold no block comments
    and no // inside string literals)."""
    h = hashlib.sha1()
    for p in sorted(glob.glob(os.path.join(ROOT, "paper_1704_08579_gb300", "csrc", "*"))):
        with open(p, encoding="utf-8") as f:
            code = [re.sub(r"//.*", "", line).rstrip() for line in f]
        h.update(os.path.basename(p).encode())
        h.update("\n".join(line for line in code if line).encode())
    return h.hexdigest()


def _profiled_traffic(name: str):
    """DRAM bytes per launch recorded from an ncu capture (profiles/<name>), or
    None when the kernel sources changed since that capture."""
    p = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(p):
        return None, None
    vals = {}
    with open(p) as f:
        for line in f:
            if ":" in line and line.strip().startswith("- "):
                k, v = line.strip()[2:].split(":", 1)
                vals[k.strip()] = v.strip().strip("`")
    if vals.get("source_sha1") != _kernel_source_sha1():
        return None, vals.get("source_sha1")
    try:
        return float(vals["dram_bytes_per_key_per_level"]), vals.get("source_sha1")
    except (KeyError, ValueError):
        return None, None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_id: str | None):
        self.proc = None
        try:
            cmd = ["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits", "-lms", "100"]
            if device_id:
                cmd += ["-i", device_id]
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, flag in zip(names, parts[5:9]):
                if flag.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _max_over_ranks(torch, value: float, world: int, device: str = "cuda") -> float:
    """The largest of every rank's `value` (the job's time is its slowest
    replica's); `device` is where the collective's tensor lives: "cuda" for
    NCCL, "cpu" for gloo."""
    if world <= 1:
        return float(value)
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def _job_gkeys_s(world: int, keys_per_rank: int, ms_per_step: float) -> float:
    """Whole-job throughput: the keys of all replicas over the slowest one's time."""
    return world * keys_per_rank / (ms_per_step / 1e3) / 1e9


def _job_e2e(torch, e2e: dict, world: int, keys_per_rank: int, device: str = "cuda") -> dict:
    """One replica's end-to-end record turned into the job's: the slowest
    replica's median step, the keys and copied bytes of all replicas."""
    if world <= 1:
        return e2e
    out = dict(e2e)
    out["ms_per_step"] = _max_over_ranks(torch, e2e["ms_per_step"], world, device)
    out["value"] = _job_gkeys_s(world, keys_per_rank, out["ms_per_step"])
    out["h2d_bytes_per_step"] = e2e["h2d_bytes_per_step"] * world
    out["d2h_bytes_per_step"] = e2e["d2h_bytes_per_step"] * world
    out["ms_min"] = out["ms_max"] = None  # per-replica extremes are not aggregated
    out["sorted"] = _max_over_ranks(torch, 0.0 if e2e["sorted"] else 1.0, world, device) == 0.0
    return out


def _device_id(torch, local_rank):
    try:
        uuid = str(torch.cuda.get_device_properties(local_rank).uuid)
        return uuid if uuid.startswith("GPU-") else "GPU-" + uuid
    except Exception:  # noqa: BLE001
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        return vis.split(",")[local_rank] if vis else str(local_rank)


def host_identity() -> dict:
    """The host the CPU baseline runs on: logical CPUs and CPU model."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() in ("Model name", "Model"):
                model = line.split(":", 1)[1].strip()
                if line.startswith("Model name"):
                    break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model and os.path.exists("/proc/cpuinfo"):
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
    import platform

    return {"nproc": os.cpu_count(), "cpu_model": model, "machine": platform.machine()}


def cpu_oracle_baseline(sample_log2: int = 24, repeats: int = 3, seed: int | None = None):
    """Times the oracle (single-threaded Appendix A quicksort) on the first
    2^sample_log2 keys of the workload's seeded stream."""
    import oracle

    n = 1 << sample_log2
    x = synth.uniform_f64(n, synth.SEEDS["c2_uniform_f64"] if seed is None else seed)
    oracle.build()
    times = []
    for _ in range(repeats):
        y = x.copy()
        t0 = time.perf_counter()
        oracle.sort_inplace(y)
        times.append(time.perf_counter() - t0)
    t = statistics.median(times)
    # Context beside it: the task-parallel form of the same oracle (identical
    # output) on every host core, same sample.
    threads = os.cpu_count() or 1
    ptimes = []
    for _ in range(repeats):
        t0 = time.perf_counter()
        oracle.sort_parallel(x, threads=threads)
        ptimes.append(time.perf_counter() - t0)
    tp = statistics.median(ptimes)
    return dict({"value": n / t / 1e9, "unit": "Gkeys/s", "cores": 1, "kind": "oracle",
                 "sample": "first 2^%d keys of the same seeded f64 stream, oracle quicksort, median of %d runs "
                           "(%.2f s each)" % (sample_log2, repeats, t),
                 "all_cores": {"value": n / tp / 1e9, "unit": "Gkeys/s", "cores": threads,
                               "kind": "task-parallel oracle (same steps, same output)"}}, **host_identity())


def run_reference(args):
    rank, world, _ = _dist_env()
    if rank != 0:
        return 0
    import oracle

    oracle.build()
    n = 1 << 22  # bounded sample per step (~0.5 s of CPU work)
    x = synth.uniform_f64(n, synth.SEEDS["c2_uniform_f64"])
    for _ in range(args.warmup):
        y = x.copy()
        oracle.sort_inplace(y)
    times = []
    for _ in range(args.steps):
        y = x.copy()
        t0 = time.perf_counter()
        oracle.sort_inplace(y)
        times.append(time.perf_counter() - t0)
    ms = 1e3 * sum(times) / len(times)
    value = n / (ms / 1e3) / 1e9
    line = {
        "impl": "reference", "metric": "Gkeys/s sorted", "value": value, "unit": "Gkeys/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": N_KEYS, "sample_n": n,
                   "note": "CPU oracle on a bounded sample of the workload (first 2^22 keys) per step"},
        "cpu_baseline": dict({"value": value, "unit": "Gkeys/s", "cores": 1, "kind": "oracle",
                              "sample": "first 2^22 keys of the workload's seeded stream per step"},
                             **host_identity()),
        "e2e": {"value": value, "unit": "Gkeys/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _time_sorts(torch, qs, bufs, stream, vals=None):
    """Sorts each buffer once on `stream`; returns (total ms, per-call stats)."""
    st = []
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        start.record(stream)
        for i, b in enumerate(bufs):
            qs.sort(b, None if vals is None else vals[i], stream=stream)
            st.append(qs.stats())
        stop.record(stream)
    stop.synchronize()
    return start.elapsed_time(stop), st


def _secondary(torch, qs, stream, name, make, steps=3, kind="f64"):
    """A short measurement of another workload (not the headline)."""
    keys = make()
    vals = None
    if isinstance(keys, tuple):
        keys, vals = keys
    n = keys.size
    dk = torch.from_numpy(keys).to("cuda")
    dv = torch.from_numpy(vals).to("cuda") if vals is not None else None
    bk = [dk.clone() for _ in range(steps + 1)]
    bv = [dv.clone() for _ in range(steps + 1)] if dv is not None else None
    del dk, dv
    torch.cuda.synchronize()  # the copies (current stream) land before the sorts (`stream`) read them
    _time_sorts(torch, qs, bk[:1], stream, None if bv is None else bv[:1])  # warm-up
    ms, st = _time_sorts(torch, qs, bk[1:], stream, None if bv is None else bv[1:])
    b = keys.itemsize + (4 if vals is not None else 0)
    ms_step = ms / steps
    drv = statistics.mean(s["ms_driver"] for s in st)
    part_bytes = statistics.mean(s["part_keys"] for s in st) * 2 * b
    out = {"workload": name, "n": n, "gkeys_s": n / (ms_step / 1e3) / 1e9, "ms_per_step": ms_step,
           "partition_kernel_gbs": part_bytes / (drv / 1e3) / 1e9 if drv > 0 else None,
           "passes_per_key": statistics.mean(s["part_keys"] for s in st) / n}
    del bk, bv
    torch.cuda.empty_cache()
    return out


def run_ours(args):
    import torch

    rank, world, local = _dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_1704_08579_gb300 as qs
    from paper_1704_08579_gb300 import build as qs_build

    if rank == 0 or world == 1:
        qs_build.build()
    if world > 1:
        torch.distributed.barrier()
    qs_build.build()
    qs.load()
    hbm_peak, peak_kind = _peaks()

    seed = synth.SEEDS["c2_uniform_f64"] + rank
    host = synth.uniform_f64(N_KEYS, seed)
    pristine = torch.from_numpy(host).to("cuda")
    total = args.warmup + args.steps
    bufs = [pristine.clone() for _ in range(total)]
    stream = torch.cuda.Stream()
    torch.cuda.synchronize()  # the copies (current stream) land before the sorts (`stream`) read them
    qs.reserve(N_KEYS, "f64")
    # Timed steps record CUDA events around the kernels only; the in-kernel
    # cycle counters (profile level 2) run on one extra, untimed sort below.
    qs.set_option("profile", 1)

    # The clock sampler starts before the warm-up so that it is producing
    # samples by the time the timed steps run.
    sampler = ClockSampler(_device_id(torch, local)) if rank == 0 else None
    _time_sorts(torch, qs, bufs[:args.warmup], stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ms, st = _time_sorts(torch, qs, bufs[args.warmup:], stream)
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    if world > 1:
        ms = _max_over_ranks(torch, ms, world)
        torch.distributed.barrier()
    # sanity: every timed output is sorted (a property check, not parity)
    for b in bufs[args.warmup:args.warmup + 2]:
        assert bool((b[1:] >= b[:-1]).all()), "benchmark output not sorted"
    del bufs
    torch.cuda.empty_cache()
    qs.set_option("profile", 2)
    extra_buf = pristine.clone()
    torch.cuda.synchronize()
    _, st_cycles = _time_sorts(torch, qs, [extra_buf], stream)
    del extra_buf
    qs.set_option("profile", 1)
    torch.cuda.empty_cache()

    ms_step = ms / args.steps
    value = _job_gkeys_s(world, N_KEYS, ms_step)
    drv_ms = statistics.mean(s["ms_driver"] for s in st)
    leaf_ms = statistics.mean(s["ms_leaf"] for s in st)
    part_keys = statistics.mean(s["part_keys"] for s in st)
    alg_bytes = part_keys * 2 * 8  # every key of a partition task read once + written once
    achieved = alg_bytes / (drv_ms / 1e3) / 1e9
    traffic_per_key_level, _ = _profiled_traffic("driver_kernel_f64_2p28.md")
    traffic = traffic_per_key_level * part_keys if traffic_per_key_level else None
    sched_bytes = (part_keys + statistics.mean(s["leaf_keys"] + s["copy_keys"] for s in st)) * 16
    line = {
        "metric": "Gkeys/s sorted", "value": value, "unit": "Gkeys/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": N_KEYS, "distribution": "uniform", "parallelism":
                   "replicas" if world > 1 else "single-gpu",
                   "l2": "inputs larger than L2: every step sorts its own 2 GiB pristine copy"},
        "roofline": {"bound": "hbm", "kernel": "driver_kernel (persistent partition passes, register tile)",
                     "achieved": achieved, "peak": hbm_peak, "peak_kind": peak_kind, "unit": "GB/s",
                     "frac": achieved / hbm_peak, "traffic": traffic,
                     "algorithmic_bytes_per_launch": alg_bytes, "kernel_ms": drv_ms,
                     "passes_per_key": part_keys / N_KEYS},
        "schedule": {"bytes_per_step": sched_bytes, "gbs_whole_step": sched_bytes / (ms_step / 1e3) / 1e9,
                     "frac_whole_step": sched_bytes / (ms_step / 1e3) / 1e9 / hbm_peak,
                     "lower_bound_1r1w_ms": 2 * 8 * N_KEYS / (hbm_peak * 1e9) * 1e3,
                     "leaf_kernel_ms": leaf_ms, "driver_kernel_ms": drv_ms,
                     "part_tasks": st[-1]["part_tasks"], "leaf_parts": st[-1]["leaf_parts"],
                     "driver_cycles_profiled_step": st_cycles[-1]["driver_cycles"]},
        "gpu_launches": 3 * args.steps,
        "clocks": clocks,
    }
    # End to end on every replica at once (each through its own host link);
    # the job's step is the slowest replica's median step.
    if world > 1:
        torch.distributed.barrier()
    e2e = _job_e2e(torch, _e2e(torch, qs, host, stream, args), world, N_KEYS)
    if rank == 0:
        line["e2e"] = e2e
        if not args.no_extra:
            line["extra"] = _extras(torch, qs, stream, hbm_peak)
            line["batched"] = _batched(torch, qs, stream)
            line["learned"] = _learned(torch, qs, stream)
        if not args.no_cpu:
            line["cpu_baseline"] = cpu_oracle_baseline()
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.barrier()
        torch.distributed.destroy_process_group()
    return 0


def _e2e(torch, qs, host, stream, args):
    """Same metric through qs_sort_host_f64: pinned host buffer in, sorted host buffer out."""
    steps = max(3, min(args.steps, 6))
    pinned = [torch.from_numpy(host).pin_memory() for _ in range(3)]
    arrs = [p.numpy() for p in pinned]
    qs.sort_host(arrs[0], stream=stream)  # warm-up (allocates the staging area)
    times = []
    for i in range(steps):
        a = arrs[1 + i % 2]
        if i >= 2:
            a[:] = host  # a fresh unsorted copy (not timed)
        t0 = time.perf_counter()
        qs.sort_host(a, stream=stream)
        times.append(time.perf_counter() - t0)
    dt = statistics.median(times)
    ok = bool(np.all(arrs[1][1:] >= arrs[1][:-1]))
    del pinned, arrs
    # The host link is shared with other jobs on the machine; the median step
    # is reported, with the fastest and slowest beside it.
    return {"value": N_KEYS / dt / 1e9, "unit": "Gkeys/s", "h2d_bytes_per_step": N_KEYS * 8,
            "d2h_bytes_per_step": N_KEYS * 8, "ms_per_step": dt * 1e3, "ms_min": min(times) * 1e3,
            "ms_max": max(times) * 1e3, "steps": steps, "sorted": ok,
            "path": "qs_sort_host_f64 on pinned (mapped) host buffers: H2D copy, sort, result written by the "
                    "leaf kernel straight into the host buffer"}


def _batched(torch, qs, stream, nseg=20_000, steps=3):
    """Batched segmented sort (20,000 int32 arrays, log-uniform sizes in [16, 2^18])
    in one graph-captured launch sequence with autotuned leaf/one-warp thresholds,
    against the plain form: one qs_sort_i32 call per array."""
    from paper_1704_08579_gb300 import autotune

    out = {}
    for kind in ("i32", "kv"):
        keys, offs = synth.segments_i32(nseg)
        n = keys.size
        dk = torch.from_numpy(keys).to("cuda")
        dv = torch.arange(n, dtype=torch.int32, device="cuda") if kind == "kv" else None
        doffs = torch.from_numpy(offs).to("cuda")
        tuned = autotune.tune(dk, doffs, dv, reps=1, use_cache=False, stream=stream)
        bk = [dk.clone() for _ in range(steps)]
        bv = [dv.clone() for _ in range(steps)] if dv is not None else None
        torch.cuda.synchronize()  # the copies land before the timed sorts on `stream` read them
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            a.record(stream)
            for i in range(steps):
                qs.sort_segmented(bk[i], doffs, None if bv is None else bv[i], stream=stream)
            b.record(stream)
        b.synchronize()
        ms_batched = a.elapsed_time(b) / steps
        ok = bool(((bk[0][1:] >= bk[0][:-1]) | (torch.isin(torch.arange(1, n, device="cuda"), doffs))).all())
        del bk, bv
        autotune.apply({})  # back to the compiled defaults for the plain form
        # Plain form: one asynchronous sort call (one launch sequence) per
        # array, no host synchronisation between them, one qs_sync_status at
        # the end; the device time spans the whole sequence.
        prof = qs.get_option("profile")
        qs.set_option("profile", 0)  # profiling would make every call synchronous
        pk = dk.clone()
        pv = dv.clone() if dv is not None else None
        bounds = offs.tolist()
        views = [(pk[bounds[i]:bounds[i + 1]], None if pv is None else pv[bounds[i]:bounds[i + 1]])
                 for i in range(nseg) if bounds[i + 1] - bounds[i] > 1]
        qs.reserve(n, kind)
        torch.cuda.synchronize()
        a2 = torch.cuda.Event(enable_timing=True)
        b2 = torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            a2.record(stream)
            for k_view, v_view in views:
                qs.sort(k_view, v_view, stream=stream, sync=False)
            b2.record(stream)
        qs.sync_status(stream)
        host_s = time.perf_counter() - t0
        b2.synchronize()
        ms_plain = a2.elapsed_time(b2)
        qs.set_option("profile", prof)
        plain_ok = bool(((pk[1:] >= pk[:-1]) | (torch.isin(torch.arange(1, n, device="cuda"), doffs))).all())
        out[kind] = {"workload": "%d %s arrays, sizes log-uniform [16, 2^18], %d keys" % (nseg, kind, n),
                     "batched_ms": ms_batched, "batched_gkeys_s": n / (ms_batched / 1e3) / 1e9,
                     "plain_per_array_ms": ms_plain, "plain_gkeys_s": n / (ms_plain / 1e3) / 1e9,
                     "plain_form": "one asynchronous qs_sort_%s call per array, one qs_sync_status at the end"
                                   % kind,
                     "plain_host_issue_ms": host_s * 1e3, "plain_sorted": plain_ok,
                     "speedup": ms_plain / ms_batched, "tuned": {k: tuned[k] for k in ("leaf_max", "small_max", "driver_items")},
                     "batched_sorted": ok}
        del dk, dv, pk, pv
        torch.cuda.empty_cache()
    return out


def _learned(torch, qs, stream, steps=3):
    """Learned-splitter form on the skewed workloads: 2^30 int32 keys Zipf(1.2)
    over 2^24 values, 2^30 int32 keys from an 8-Gaussian mixture, 2^28 FP64
    keys lognormal(0, 2).  The network is first trained (untimed) on
    sort-generated pairs with the library's kernels; then the plain sort, the
    bucket form with sampled splitters and the learned form (two bucket
    levels, the default; and again with one level) are timed on the same
    array (median of `steps`), and the bucket forms' outputs are checked
    equal to the plain sort's."""
    import synth.device as sdev
    from paper_1704_08579_gb300 import learned

    models, train_s = {}, {}
    for kind in ("i32", "f64"):
        t0 = time.perf_counter()
        X, T = learned.training_set(kind, 4096, 1 << 16, seed=7)
        models[kind], _ = learned.train(X, T, steps=3000, batch=128, lr=3e-4, seed=3)
        torch.cuda.synchronize()
        train_s[kind] = time.perf_counter() - t0
        del X, T
    out = {"train_seconds": train_s}
    cases = (("zipf_i32_2^30", "i32", lambda: sdev.zipf_i32(1 << 30)),
             ("gauss_mix8_i32_2^30", "i32", lambda: sdev.gauss_mix_i32(1 << 30)),
             ("lognormal_f64_2^28", "f64", lambda: sdev.lognormal_f64(1 << 28)))
    for name, kind, make in cases:
        pristine = make()
        n = pristine.numel()
        work = torch.empty_like(pristine)
        ref = None
        res = {}
        for arm in ("plain", "sampled", "learned", "sampled_1level", "learned_1level"):
            qs.set_option("bucket_levels", 1 if arm.endswith("_1level") else 0)
            times, st = [], None
            for r in range(steps + 1):
                work.copy_(pristine)
                torch.cuda.synchronize()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                with torch.cuda.stream(stream):
                    a.record(stream)
                    if arm == "plain":
                        qs.sort(work, stream=stream)
                    else:
                        qs.sort_learned(work, models[kind] if arm.startswith("learned") else None, stream=stream)
                    b.record(stream)
                b.synchronize()
                st = qs.stats()
                if r:
                    times.append(a.elapsed_time(b))
            ms = statistics.median(times)
            res[arm] = {"ms": ms, "gkeys_s": n / (ms / 1e3) / 1e9}
            if arm == "plain":
                ref = work.clone()
                res[arm]["sorted"] = bool((ref[1:] >= ref[:-1]).all())
            else:
                res[arm].update({"imbalance_err": st["bucket_dev"] / (2.0 * n * 256),
                                 "bucket_max_over_even": st["bucket_max"] / (n / 256.0),
                                 "buckets_over_bound": st["bucket_over"],
                                 "equal_to_plain": bool(torch.equal(work.view(torch.int64) if kind == "f64" else work,
                                                                    ref.view(torch.int64) if kind == "f64" else ref))})
        qs.set_option("bucket_levels", 0)
        res["n"] = n
        res["bucket_levels"] = {"sampled": 2, "learned": 2, "sampled_1level": 1, "learned_1level": 1}
        out[name] = res
        del pristine, work, ref
        torch.cuda.empty_cache()
    return out


def _leaf_sweep(torch, qs, stream, total=1 << 24, reps=3):
    """Many independent arrays of one size n in one segmented-sort call, for n
    from 2 up past the leaf threshold: the leaf network's throughput per array
    size (and where the partition path takes over)."""
    out = {}
    sizes = [2, 8, 32, 100, 512, 513, 1000, 2048, 3000, 4096, 6000, 8192, 12000, 16384, 65536]
    for kind, dtype in (("i32", torch.int32), ("f64", torch.float64)):
        rows = []
        for n in sizes:
            nseg = max(1, total // n)
            m = nseg * n
            if dtype == torch.int32:
                keys = torch.from_numpy(synth.uniform_i32(m, 0x1EAF)).to("cuda")
            else:
                keys = torch.from_numpy(synth.uniform_f64(m, 0x1EAF)).to("cuda")
            offs = torch.arange(0, nseg + 1, dtype=torch.int64, device="cuda") * n
            work = torch.empty_like(keys)
            times = []
            for r in range(reps + 1):
                work.copy_(keys)
                torch.cuda.synchronize()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                with torch.cuda.stream(stream):
                    a.record(stream)
                    qs.sort_segmented(work, offs, stream=stream)
                    b.record(stream)
                b.synchronize()
                if r:
                    times.append(a.elapsed_time(b))
            ms = statistics.median(times)
            rows.append({"n": n, "arrays": nseg, "ms": ms, "gkeys_s": m / (ms / 1e3) / 1e9,
                         "ns_per_array": ms * 1e6 / nseg})
            del keys, work, offs
        out[kind] = rows
    torch.cuda.empty_cache()
    return out


def _extras(torch, qs, stream, hbm_peak):
    out = []
    n = N_KEYS
    args_log2n = n.bit_length() - 1
    out.append(_secondary(torch, qs, stream, "f64 sorted 2^%d" % args_log2n, lambda: synth.f64_config("sorted", n)))
    out.append(_secondary(torch, qs, stream, "f64 reverse 2^%d" % args_log2n, lambda: synth.f64_config("reverse", n)))
    out.append(_secondary(torch, qs, stream, "f64 16-unique 2^%d" % args_log2n, lambda: synth.f64_config("few", n)))
    out.append(_secondary(torch, qs, stream, "i32 uniform 2^%d" % args_log2n, lambda: synth.uniform_i32(n, 0x5EED0001)))
    out.append(_secondary(torch, qs, stream, "kv uniform 2^%d" % args_log2n, lambda: synth.kv_config("uniform", n)))
    # qs_partition_f64 alone with the true median as pivot.
    x = synth.f64_config("uniform", n)
    pivot = float(np.partition(x, n // 2)[n // 2])
    d = torch.from_numpy(x).to("cuda")
    bufs = [d.clone() for _ in range(4)]
    del d
    torch.cuda.synchronize()  # the copies land before the partitions on `stream` read them
    ms_k, ms_t, split = [], [], None
    with torch.cuda.stream(stream):
        for i, b in enumerate(bufs):
            split = qs.partition(b, pivot, stream=stream)
            s = qs.stats()
            if i:
                ms_k.append(s["ms_driver"])
                ms_t.append(s["ms_total"])
    km, tm = statistics.mean(ms_k), statistics.mean(ms_t)
    out.append({"workload": "qs_partition_f64 2^%d, pivot = true median" % args_log2n, "n": n, "split": split,
                "kernel_ms": km, "kernel_gbs": 16 * n / (km / 1e3) / 1e9,
                "kernel_frac": 16 * n / (km / 1e3) / 1e9 / hbm_peak,
                "call_ms_with_copy_back": tm, "call_gkeys_s": n / (tm / 1e3) / 1e9})
    del bufs
    torch.cuda.empty_cache()
    return out


def run_partition_only(args):
    """qs_partition_f64 alone on the uniform input with the true median as pivot
    (one JSON line with the per-phase cycle breakdown); used for profiling."""
    import torch

    import paper_1704_08579_gb300 as qs
    from paper_1704_08579_gb300 import build as qs_build

    qs_build.build()
    x = synth.f64_config("uniform", N_KEYS)
    pivot = float(np.partition(x, N_KEYS // 2)[N_KEYS // 2])
    # One device copy of the input, restored from pinned host memory before
    # every call (not timed): the device holds the input plus the library's
    # scratch, nothing else.
    pristine = torch.from_numpy(x).pin_memory()
    d = torch.empty(N_KEYS, dtype=torch.float64, device="cuda")
    qs.reserve(N_KEYS, "f64")
    qs.set_option("profile", 1)
    stream = torch.cuda.Stream()
    res = []
    calls = args.warmup + args.steps + 1
    with torch.cuda.stream(stream):
        for i in range(calls):
            d.copy_(pristine, non_blocking=True)
            if i == calls - 1:
                qs.set_option("profile", 2)  # cycle counters on the last, untimed call only
            split = qs.partition(d, pivot, stream=stream)
            if args.warmup <= i < calls - 1:
                res.append(qs.stats())
        cycles = qs.stats()["driver_cycles"]
    qs.set_option("profile", 1)
    km = statistics.mean(r["ms_driver"] for r in res)
    print(json.dumps({"op": "partition", "n": N_KEYS, "split": split, "kernel_ms": km,
                      "kernel_gbs": 16 * N_KEYS / (km / 1e3) / 1e9,
                      "driver_cycles": cycles, "grid": res[-1]["grid_driver"]}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-extra", action="store_true", help="skip the secondary workloads")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--op", choices=["sort", "partition", "learned", "batched", "leafsweep"], default="sort",
                    help="partition / learned / batched: that measurement alone (not the benchmark line)")
    ap.add_argument("--log2n", type=int, default=LOG2N,
                    help="log2 of the keys per sort (28 = the benchmark workload; smaller only for profiling)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)  # at least three untimed warm-up steps
    global N_KEYS, WORKLOAD
    N_KEYS = 1 << args.log2n
    WORKLOAD = WORKLOAD % args.log2n
    if args.impl == "reference":
        return run_reference(args)
    if args.op == "partition":
        return run_partition_only(args)
    if args.op in ("learned", "batched", "leafsweep"):
        return run_section(args.op)
    return run_ours(args)


def run_section(name: str) -> int:
    """One secondary measurement alone, printed as its own JSON line."""
    import torch

    import paper_1704_08579_gb300 as qs
    from paper_1704_08579_gb300 import build as qs_build

    torch.cuda.set_device(0)
    qs_build.build()
    qs.load()
    stream = torch.cuda.Stream()
    res = {"learned": _learned, "batched": _batched, "leafsweep": _leaf_sweep}[name](torch, qs, stream)
    print(json.dumps({"section": name, name: res}), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
