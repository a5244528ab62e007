"""GPU parity of qs_sort_{i32,f64,kv} against the oracle (Appendix A / Sections
III-A..III-D).  Keys must be bit-identical to the oracle's; for key/value
pairs each run of equal keys must hold the same multiset of values.

Sizes cover the single-warp leaf (<= 512), the merge-path group leaf (<= 32768
i32, <= 16384 f64/kv; groups of any multiple of 32 threads, so run counts that
are not powers of two), several device-wide partition levels, ragged tails,
duplicate-heavy and all-equal inputs, extreme keys and unaligned pointers.
"""
import numpy as np
import pytest

import synth
from qs_testutil import assert_keys_equal, assert_kv_sorted_equal, oracle_sort, qs_gpu, to_dev

pytestmark = pytest.mark.gpu

SIZES = [2, 3, 31, 32, 33, 100, 511, 512, 513, 1000, 1025, 1536, 2049, 3000, 4095, 4096, 4097, 7_000, 8191, 8192,
         8193, 12_345, 16_383, 16_384, 16_385, 23_457, 32_767, 32_768, 32_769, 65_543, 300_001]


def _sort_dev(qs, x, v=None, koff=0, voff=0):
    import torch

    n = x.size
    kbuf = to_dev(np.concatenate([np.zeros(koff, x.dtype), x]))
    d = kbuf[koff:koff + n]
    if v is not None:
        vbuf = to_dev(np.concatenate([np.zeros(voff, np.int32), v]))
        dv = vbuf[voff:voff + n]
        qs.sort(d, dv)
        torch.cuda.synchronize()
        return d.cpu().numpy(), dv.cpu().numpy()
    qs.sort(d)
    torch.cuda.synchronize()
    return d.cpu().numpy()


@pytest.mark.parametrize("n", SIZES)
def test_sort_i32_sizes(n):
    qs = qs_gpu()
    x = synth.uniform_i32(n, 300 + n)
    assert_keys_equal(_sort_dev(qs, x), oracle_sort(x))


@pytest.mark.parametrize("n", SIZES)
def test_sort_f64_sizes(n):
    qs = qs_gpu()
    x = synth.uniform_f64(n, 400 + n)
    assert_keys_equal(_sort_dev(qs, x), oracle_sort(x))


@pytest.mark.parametrize("n", SIZES)
def test_sort_kv_sizes(n):
    qs = qs_gpu()
    k, v = synth.kv_config("uniform", n, 500 + n)
    gk, gv = _sort_dev(qs, k, v)
    ok, ov = oracle_sort(k, v)
    assert_kv_sorted_equal(k, v, gk, gv, ok, ov)


def test_sort_i32_config_small():
    """Single sort of one int32 array, n = 2^20, keys uniform over the full range."""
    qs = qs_gpu()
    x = synth.uniform_i32(1 << 20, synth.SEEDS["c1_uniform_i32"])
    assert_keys_equal(_sort_dev(qs, x), oracle_sort(x))


@pytest.mark.parametrize("dist", ["uniform", "sorted", "reverse", "few"])
def test_sort_f64_distributions(dist):
    qs = qs_gpu()
    x = synth.f64_config(dist, 1 << 20)
    assert_keys_equal(_sort_dev(qs, x), oracle_sort(x))


@pytest.mark.parametrize("dist", ["uniform", "mod1000", "sorted", "reverse"])
def test_sort_kv_distributions(dist):
    qs = qs_gpu()
    k, v = synth.kv_config(dist, 1 << 20)
    gk, gv = _sort_dev(qs, k, v)
    ok, ov = oracle_sort(k, v)
    assert_kv_sorted_equal(k, v, gk, gv, ok, ov)
    np.testing.assert_array_equal(k[gv], gk)  # value = original index: each pair intact


@pytest.mark.parametrize("n", [100, 5000, 100_000, 1 << 20])
def test_sort_duplicates(n):
    qs = qs_gpu()
    cases = [np.full(n, 7, np.int32), synth.mod_i32(n, 3, 2), synth.mod_i32(n, 4, 3) - 1,
             np.where(synth.mod_i32(n, 5, 4) == 0, 2**31 - 1, synth.uniform_i32(n, 6)).astype(np.int32),
             np.where(synth.mod_i32(n, 7, 3) == 0, -2**31, 2**31 - 1).astype(np.int32)]
    for x in cases:
        assert_keys_equal(_sort_dev(qs, x), oracle_sort(x))


@pytest.mark.parametrize("n", [500, 4096, 70_000])
def test_sort_kv_largest_keys(n):
    """Keys equal to the padding key must keep their own values (Section III-A-3 padding)."""
    qs = qs_gpu()
    k = np.where(synth.mod_i32(n, 9, 3) == 0, 2**31 - 1, synth.mod_i32(n, 10, 50)).astype(np.int32)
    v = np.arange(n, dtype=np.int32)
    gk, gv = _sort_dev(qs, k, v)
    ok, ov = oracle_sort(k, v)
    assert_kv_sorted_equal(k, v, gk, gv, ok, ov)
    np.testing.assert_array_equal(k[gv], gk)


def test_sort_f64_infinities():
    qs = qs_gpu()
    n = 50_000
    x = synth.uniform_f64(n, 12)
    sel = synth.mod_i32(n, 13, 10)
    x = np.where(sel == 0, np.inf, np.where(sel == 1, -np.inf, x))
    assert_keys_equal(_sort_dev(qs, x), oracle_sort(x))


@pytest.mark.parametrize("n", [3000, 50_000, 1 << 20])
def test_sort_f64_extremes(n):
    """FP64 keys at the ends of the bit-pattern order the integer compares rely
    on: +-DBL_MAX, +-smallest normal, +-subnormals, +-1, mixed into uniform
    keys; an all-equal array; an array of only two subnormals."""
    qs = qs_gpu()
    fi = np.finfo(np.float64)
    special = np.array([fi.max, -fi.max, fi.tiny, -fi.tiny, 5e-324, -5e-324, 2.5e-310, -2.5e-310, 1.0, -1.0])
    sel = synth.mod_i32(n, 21, 2 * special.size)
    x = synth.uniform_f64(n, 22)
    x = np.where(sel < special.size, special[np.minimum(sel, special.size - 1)], x)
    assert_keys_equal(_sort_dev(qs, x), oracle_sort(x))
    y = np.full(n, -3.75)
    assert_keys_equal(_sort_dev(qs, y), oracle_sort(y))
    z = np.where(synth.mod_i32(n, 23, 2) == 0, 5e-324, -5e-324)
    assert_keys_equal(_sort_dev(qs, z), oracle_sort(z))


@pytest.mark.parametrize("koff,voff", [(1, 1), (1, 2), (3, 0), (2, 2)])
def test_sort_unaligned(koff, voff):
    qs = qs_gpu()
    n = 100_003
    x = synth.uniform_i32(n, 14)
    assert_keys_equal(_sort_dev(qs, x, koff=koff), oracle_sort(x))
    y = synth.uniform_f64(n, 15)
    assert_keys_equal(_sort_dev(qs, y, koff=koff % 2), oracle_sort(y))
    k, v = synth.kv_config("mod1000", n, 16)
    gk, gv = _sort_dev(qs, k, v, koff=koff, voff=voff)
    ok, ov = oracle_sort(k, v)
    assert_kv_sorted_equal(k, v, gk, gv, ok, ov)


def test_sort_workspace_reuse():
    """Grow, shrink and alternate kinds: the workspace is reused across calls."""
    qs = qs_gpu()
    for n in (1 << 18, 1000, 1 << 19, 77_777, 1 << 16):
        x = synth.uniform_i32(n, n)
        assert_keys_equal(_sort_dev(qs, x), oracle_sort(x))
        y = synth.uniform_f64(n, n + 1)
        assert_keys_equal(_sort_dev(qs, y), oracle_sort(y))


def test_sort_host_buffers():
    qs = qs_gpu()
    x = synth.uniform_f64(200_001, 17)
    h = x.copy()
    qs.sort_host(h)
    assert_keys_equal(h, oracle_sort(x))
    k, v = synth.kv_config("uniform", 100_001, 18)
    hk, hv = k.copy(), v.copy()
    qs.sort_host(hk, hv)
    ok, ov = oracle_sort(k, v)
    assert_kv_sorted_equal(k, v, hk, hv, ok, ov)


def _pinned(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()


@pytest.mark.parametrize("n", [2, 5000, 200_001, (1 << 20) + 3])
def test_sort_host_pinned_buffers(n):
    """Pinned (mapped) host buffers: the leaf kernel writes the sorted parts
    straight into them, and finished runs of equal keys are copied out from
    whichever buffer they were finished in.  Uniform, 16-distinct and
    all-equal FP64 keys, int32 keys with 7 distinct values, key/value pairs
    with 1000 distinct keys, against the oracle."""
    qs = qs_gpu()
    cases = [synth.uniform_f64(n, 30), synth.f64_config("few", n, 31), np.full(n, 2.5),
             synth.mod_i32(n, 32, 7)]
    for x in cases:
        h = _pinned(x)
        qs.sort_host(h)
        assert_keys_equal(h, oracle_sort(x))
    k, v = synth.kv_config("mod1000", n, 33)
    hk, hv = _pinned(k), _pinned(v)
    qs.sort_host(hk, hv)
    ok, ov = oracle_sort(k, v)
    assert_kv_sorted_equal(k, v, hk, hv, ok, ov)


def test_wait_limit_reports_timeout_and_recovers():
    """A device-side wait that runs out ends the kernel with QS_ERR_TIMEOUT
    (no hang, no fault); the next call works."""
    qs = qs_gpu()
    x = synth.uniform_i32(1 << 20, 19)
    qs.set_option("wait_limit_ns", 0)
    try:
        with pytest.raises(qs.QSError) as e:
            _sort_dev(qs, x)
        assert e.value.code == -5
    finally:
        qs.set_option("wait_limit_ns", 2_000_000_000)
    assert_keys_equal(_sort_dev(qs, x), oracle_sort(x))


def test_capacity_overflow_reported_and_recovers():
    qs = qs_gpu()
    x = synth.uniform_i32(1 << 20, 20)
    qs.set_option("task_cap", 1)
    try:
        with pytest.raises(qs.QSError) as e:
            _sort_dev(qs, x)
        assert e.value.code == -6
    finally:
        qs.set_option("task_cap", 0)
    assert_keys_equal(_sort_dev(qs, x), oracle_sort(x))


@pytest.mark.parametrize("kind,items", [("i32", 16), ("i32", 32), ("f64", 8), ("f64", 16), ("f64", 20), ("kv", 8),
                                        ("kv", 16), ("kv", 20)])
def test_narrow_tile_variant(kind, items):
    """Every partition tile variant chosen explicitly (QS_OPT_DRIVER_ITEMS:
    narrow and wide prefetched tiles, and the register tile loaded without a
    prefetch buffer: 32 keys per thread for int32, 20 for FP64 and key/value) gives the
    same results: sorts of several sizes and distributions, and a partition
    (which otherwise uses its own default tile)."""
    import torch

    import oracle

    qs = qs_gpu()
    qs.set_option("driver_items", items)
    try:
        for n, seed in ((8193, 1), (300_001, 2), ((1 << 20) + 7, 3)):
            if kind == "i32":
                for x in (synth.uniform_i32(n, seed), synth.mod_i32(n, seed, 1000)):
                    assert_keys_equal(_sort_dev(qs, x), oracle_sort(x))
            elif kind == "f64":
                for dist in ("uniform", "few", "reverse"):
                    x = synth.f64_config(dist, n, seed)
                    assert_keys_equal(_sort_dev(qs, x), oracle_sort(x))
            else:
                k, v = synth.kv_config("mod1000", n, seed)
                gk, gv = _sort_dev(qs, k, v)
                ok, ov = oracle_sort(k, v)
                assert_kv_sorted_equal(k, v, gk, gv, ok, ov)
        n = (1 << 20) + 5
        x = synth.uniform_f64(n, 9) if kind == "f64" else synth.uniform_i32(n, 9)
        pivot = x[n // 3]
        if kind == "kv":
            v = np.arange(n, dtype=np.int32)
            dk, dv = to_dev(x), to_dev(v)
            split = qs.partition(dk, int(pivot), dv)
            esplit, ek, ev = oracle.partition(x, int(pivot), v)
            torch.cuda.synchronize()
            assert split == esplit
            assert_keys_equal(dk.cpu().numpy(), ek)
            np.testing.assert_array_equal(dv.cpu().numpy(), ev)
        else:
            d = to_dev(x)
            split = qs.partition(d, pivot)
            esplit, ek = oracle.partition(x, pivot)
            torch.cuda.synchronize()
            assert split == esplit
            assert_keys_equal(d.cpu().numpy(), ek)
    finally:
        qs.set_option("driver_items", 0)


@pytest.mark.parametrize("kind", ["i32", "f64", "kv"])
def test_ordered_and_unordered_placement(kind):
    """Both placements of a sort's partition tiles (QS_OPT_ORDERED) give the
    oracle's keys: tiles claiming their output ranges with atomics (default)
    and tiles placed in input order by the look-back."""
    qs = qs_gpu()
    try:
        for ordered in (1, 0):
            qs.set_option("ordered", ordered)
            for n, seed in ((70_001, 31), ((1 << 21) + 3, 32)):
                if kind == "i32":
                    for x in (synth.uniform_i32(n, seed), synth.mod_i32(n, seed, 7)):
                        assert_keys_equal(_sort_dev(qs, x), oracle_sort(x))
                elif kind == "f64":
                    for dist in ("uniform", "sorted", "few"):
                        x = synth.f64_config(dist, n, seed)
                        assert_keys_equal(_sort_dev(qs, x), oracle_sort(x))
                else:
                    for dist in ("uniform", "mod1000"):
                        k, v = synth.kv_config(dist, n, seed)
                        gk, gv = _sort_dev(qs, k, v)
                        ok, ov = oracle_sort(k, v)
                        assert_kv_sorted_equal(k, v, gk, gv, ok, ov)
    finally:
        qs.set_option("ordered", 0)


@pytest.mark.parametrize("kind", ["i32", "f64", "kv"])
def test_small_leaf_thresholds(kind):
    """Run-time leaf / one-warp thresholds down to the minimum (32): the
    recursion then reaches partition tasks of 33 keys, whose tiles are
    nearly all ragged edges, and deep trees of tiny tasks -- with both tile
    placements.  Keys against the oracle (key/value: value multisets per run
    of equal keys)."""
    qs = qs_gpu()
    try:
        for leaf, small in ((32, 32), (64, 32), (512, 64), (2048, 256), (8192, 512)):
            qs.set_option("leaf_max", leaf)
            qs.set_option("small_max", small)
            for ordered in (0, 1):
                qs.set_option("ordered", ordered)
                for n, seed in ((30_011, 41), (200_003, 42)):
                    if kind == "i32":
                        for x in (synth.uniform_i32(n, seed), synth.mod_i32(n, seed, 7)):
                            assert_keys_equal(_sort_dev(qs, x), oracle_sort(x))
                    elif kind == "f64":
                        for dist in ("uniform", "few", "reverse"):
                            x = synth.f64_config(dist, n, seed)
                            assert_keys_equal(_sort_dev(qs, x), oracle_sort(x))
                    else:
                        for dist in ("uniform", "mod1000"):
                            k, v = synth.kv_config(dist, n, seed)
                            gk, gv = _sort_dev(qs, k, v)
                            ok, ov = oracle_sort(k, v)
                            assert_kv_sorted_equal(k, v, gk, gv, ok, ov)
    finally:
        qs.set_option("leaf_max", 0)
        qs.set_option("small_max", 0)
        qs.set_option("ordered", 0)
