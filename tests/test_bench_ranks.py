"""Host logic of bench.py's multi-replica run, on CPU: two gloo ranks.

With N > 1 the benchmark runs one replica per GPU (weak scaling; no
collective on the data path): the job's time is the slowest replica's, its
value counts the keys of every replica, and the end-to-end record is
aggregated the same way.  The reference arm runs on rank 0 only; the other
ranks leave at once.  These tests exercise exactly those helpers over a real
gloo process group (rendezvous on 127.0.0.1).
"""
import argparse
import os
import socket

import pytest

import bench


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch
    import torch.distributed as dist

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = (7.0, 11.5)[rank]
        slowest = bench._max_over_ranks(torch, ms, world, device="cpu")
        value = bench._job_gkeys_s(world, 1 << 28, slowest)
        rec = {"value": 1.0, "ms_per_step": (30.0, 42.0)[rank], "ms_min": 1.0, "ms_max": 2.0,
               "h2d_bytes_per_step": 8 << 28, "d2h_bytes_per_step": 8 << 28, "sorted": rank == 0}
        job = bench._job_e2e(torch, rec, world, 1 << 28, device="cpu")
        q.put((rank, bench._dist_env(), slowest, value, job))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_replica_and_count_every_key():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    try:
        got = sorted(q.get(timeout=180) for _ in procs)
    finally:
        for p in procs:
            p.join(timeout=60)
            if p.is_alive():
                p.kill()
    assert [p.exitcode for p in procs] == [0, 0]
    for rank, env, slowest, value, job in got:
        assert env == (rank, 2, rank)
        assert slowest == 11.5
        assert value == pytest.approx(2 * (1 << 28) / 11.5e-3 / 1e9)
        assert job["ms_per_step"] == 42.0
        assert job["value"] == pytest.approx(2 * (1 << 28) / 42.0e-3 / 1e9)
        assert job["h2d_bytes_per_step"] == job["d2h_bytes_per_step"] == 2 * (8 << 28)
        assert job["ms_min"] is None and job["ms_max"] is None
        assert job["sorted"] is False  # one replica's output was not sorted: the job's is not


def test_single_replica_records_pass_through():
    rec = {"value": 3.0, "ms_per_step": 5.0, "sorted": True}
    assert bench._job_e2e(None, rec, 1, 1 << 28) is rec
    assert bench._max_over_ranks(None, 4.5, 1) == 4.5
    assert bench._job_gkeys_s(1, 1 << 28, 1000.0) == pytest.approx((1 << 28) / 1e9)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    assert bench.run_reference(argparse.Namespace(steps=1, warmup=3)) == 0
    assert capsys.readouterr().out == ""


def test_reference_arm_line_on_rank_zero(monkeypatch, capsys):
    """Rank 0 prints one JSON line with the contract's keys: the oracle's
    throughput on its bounded sample, the same figure as its cpu_baseline and
    as its end-to-end value (no host-device copies)."""
    import json
    import sys

    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    # main() formats these module globals; restore them afterwards.
    monkeypatch.setattr(bench, "WORKLOAD", bench.WORKLOAD)
    monkeypatch.setattr(bench, "N_KEYS", bench.N_KEYS)
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--steps", "1", "--warmup", "3"])
    assert bench.main() == 0
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["n_gpus"] == 1 and d["steps"] == 1 and d["warmup"] == 3
    assert d["higher_is_better"] is True and d["dtype"] == "f64" and d["value"] > 0
    assert d["config"]["workload"].startswith("f64 sort, n=2^28") and d["config"]["n"] == 1 << 28
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == d["value"] and cb["sample"]
    assert cb["nproc"] >= 1 and "cpu_model" in cb
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
