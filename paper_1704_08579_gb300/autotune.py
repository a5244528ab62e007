"""Autotuner for the run-time knobs of the sort: the leaf threshold (largest
part handed to the leaf kernel, QS_OPT_LEAF_MAX), the one-warp threshold
(QS_OPT_SMALL_MAX) and the keys per thread of a partition tile
(QS_OPT_DRIVER_ITEMS, one of the compiled tile variants).  Each candidate
is timed on the caller's own data with CUDA events (a fresh copy of the input
per run, so every run sorts the same unsorted data); the fastest is kept,
applied with qs_set_option, and recorded in a JSON cache keyed by GPU name and
workload signature.
"""
from __future__ import annotations

import json
import os
import statistics

import paper_1704_08579_gb300 as qs

HERE = os.path.dirname(os.path.abspath(__file__))
CACHE_DIR = os.path.join(HERE, "tuning")

# The last choice of each kind hands parts of up to twice the shared-memory
# size to the leaf kernel, which then splits them once itself.
LEAF_CHOICES = {"i32": (8192, 16384, 32768, 65536), "f64": (4096, 8192, 16384, 32768), "kv": (4096, 8192, 16384, 32768)}
SMALL_CHOICES = (128, 256, 512)
ITEMS_CHOICES = {"i32": (32, 16), "f64": (20, 16, 8), "kv": (20, 16, 8)}  # the kind's sort default first


def _cache_path(gpu_name: str) -> str:
    safe = "".join(ch if ch.isalnum() else "_" for ch in gpu_name)
    return os.path.join(CACHE_DIR, safe + ".json")


def _load_cache(gpu_name: str) -> dict:
    p = _cache_path(gpu_name)
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f)
    return {}


def _store_cache(gpu_name: str, cache: dict) -> None:
    os.makedirs(CACHE_DIR, exist_ok=True)
    tmp = _cache_path(gpu_name) + ".tmp%d" % os.getpid()
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, _cache_path(gpu_name))


def signature(kind: str, n: int, nseg: int) -> str:
    """Workload key: kind, log2 of the key count, log2 of the segment count."""
    return "%s:n2^%d:seg2^%d" % (kind, max(n, 1).bit_length() - 1, max(nseg, 1).bit_length() - 1)


def cached_entry(cache: dict, sig: str, kind: str):
    """The cached choice for `sig`, or None when there is none or it names a
    value outside the current candidate lists (a cache written by a library
    whose tile variants or thresholds differed: the tile selector values
    change with the compiled variants, so such an entry is tuned again)."""
    e = cache.get(sig)
    if not isinstance(e, dict):
        return None
    ok = (e.get("leaf_max") in LEAF_CHOICES[kind] and e.get("small_max") in SMALL_CHOICES
          and e.get("driver_items") in ITEMS_CHOICES[kind])
    return e if ok else None


def apply(cfg: dict) -> None:
    qs.set_option("leaf_max", int(cfg.get("leaf_max", 0)))
    qs.set_option("small_max", int(cfg.get("small_max", 0)))
    qs.set_option("driver_items", int(cfg.get("driver_items", 0)))


def tune(keys, offsets=None, values=None, reps: int = 2, use_cache: bool = True, stream=None) -> dict:
    """Tunes (leaf_max, small_max, driver_items) for sorting `keys` (CUDA
    tensor), segmented by `offsets` if given; returns {"leaf_max", "small_max",
    "driver_items", "ms", "table"} and leaves the winner applied.  The input
    tensors are not modified."""
    import torch

    kind = "kv" if values is not None else ("i32" if keys.dtype == torch.int32 else "f64")
    nseg = 1 if offsets is None else offsets.numel() - 1
    gpu = torch.cuda.get_device_name()
    sig = signature(kind, keys.numel(), nseg)
    cache = _load_cache(gpu) if use_cache else {}
    hit = cached_entry(cache, sig, kind) if use_cache else None
    if hit is not None:
        apply(hit)
        return dict(hit, cached=True)
    stream = stream or torch.cuda.current_stream()
    # The inputs were written on the caller's current stream: order `stream` after them.
    stream.wait_stream(torch.cuda.current_stream())
    work_k = torch.empty_like(keys)
    work_v = torch.empty_like(values) if values is not None else None
    table = []

    def timed(cfg):
        apply(cfg)
        times = []
        for _ in range(reps + 1):  # the first run warms up (and captures the graph)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            with torch.cuda.stream(stream):
                # The fresh copy goes on the sort's own stream, so the sort
                # starts only once its input has landed.
                work_k.copy_(keys)
                if work_v is not None:
                    work_v.copy_(values)
                a.record(stream)
                if offsets is None:
                    qs.sort(work_k, work_v, stream=stream)
                else:
                    qs.sort_segmented(work_k, offsets, work_v, stream=stream)
                b.record(stream)
            b.synchronize()
            times.append(a.elapsed_time(b))
        row = dict(cfg, ms=statistics.median(times[1:]))
        table.append(row)
        return row

    # Thresholds with the kind's default sort tile, then the other tile variants at the best thresholds.
    for leaf in LEAF_CHOICES[kind]:
        for small in SMALL_CHOICES:
            if small <= leaf:
                timed({"leaf_max": leaf, "small_max": small, "driver_items": ITEMS_CHOICES[kind][0]})
    best = min(table, key=lambda r: r["ms"])
    for items in ITEMS_CHOICES[kind][1:]:
        timed({"leaf_max": best["leaf_max"], "small_max": best["small_max"], "driver_items": items})
    best = min(table, key=lambda r: r["ms"])
    result = {"leaf_max": best["leaf_max"], "small_max": best["small_max"], "driver_items": best["driver_items"],
              "ms": best["ms"], "table": table}
    apply(result)
    if use_cache:
        cache[sig] = {k: result[k] for k in ("leaf_max", "small_max", "driver_items", "ms")}
        _store_cache(gpu, cache)
    return result
