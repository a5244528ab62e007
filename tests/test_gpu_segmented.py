"""GPU parity of the batched (segmented) sort, qs_sort_segmented_{i32,f64,kv}:
every segment must equal the oracle's sort of that segment (keys bit-exact;
key/value: equal-key runs as value multisets), for segments of log-uniform
sizes spanning warp leaves, CTA leaves and multi-level partitions, plus the
edge cases (empty and single-key segments, one segment = whole array, no
segments, a bad offset table), graph replay with new data in the same
buffers, and the full 20,000-segment workload with sampled segment checks.
"""
import numpy as np
import pytest

import oracle
import synth
from qs_testutil import assert_keys_equal, assert_kv_sorted_equal, qs_gpu, to_dev

pytestmark = pytest.mark.gpu


def _segments(nseg, seed, lo=16, hi=1 << 14):
    sizes = synth.segment_sizes(nseg, seed, lo, hi)
    offs = np.zeros(nseg + 1, dtype=np.int64)
    np.cumsum(sizes, out=offs[1:])
    return offs


def _check_segments(x, got, offs, segs=None, vals_in=None, vals_out=None):
    idx = range(len(offs) - 1) if segs is None else segs
    for i in idx:
        a, b = int(offs[i]), int(offs[i + 1])
        if vals_in is None:
            assert_keys_equal(got[a:b], oracle.sort(x[a:b]))
        else:
            ok, ov = oracle.sort(x[a:b], vals_in[a:b])
            assert_kv_sorted_equal(x[a:b], vals_in[a:b], got[a:b], vals_out[a:b], ok, ov)


@pytest.mark.parametrize("kind", ["i32", "f64"])
def test_segmented_keys(kind):
    import torch

    qs = qs_gpu()
    offs = _segments(300, 41)
    n = int(offs[-1])
    x = synth.uniform_i32(n, 42) if kind == "i32" else synth.uniform_f64(n, 43)
    d = to_dev(x)
    qs.sort_segmented(d, to_dev(offs))
    torch.cuda.synchronize()
    _check_segments(x, d.cpu().numpy(), offs)


def test_segmented_kv():
    import torch

    qs = qs_gpu()
    offs = _segments(200, 44)
    n = int(offs[-1])
    k = synth.mod_i32(n, 45, 300)
    v = np.arange(n, dtype=np.int32)
    dk, dv = to_dev(k), to_dev(v)
    qs.sort_segmented(dk, to_dev(offs), dv)
    torch.cuda.synchronize()
    _check_segments(k, dk.cpu().numpy(), offs, vals_in=v, vals_out=dv.cpu().numpy())


def test_segmented_edge_cases():
    import torch

    qs = qs_gpu()
    sizes = [0, 1, 2, 0, 513, 4096, 4097, 100_000, 1, 0, 31, 70_000, 0]
    offs = np.zeros(len(sizes) + 1, dtype=np.int64)
    np.cumsum(sizes, out=offs[1:])
    n = int(offs[-1])
    x = synth.mod_i32(n, 46, 7)  # heavy duplicates
    d = to_dev(x)
    qs.sort_segmented(d, to_dev(offs))
    torch.cuda.synchronize()
    _check_segments(x, d.cpu().numpy(), offs)
    # one segment covering everything equals a plain sort
    y = synth.uniform_f64(200_001, 47)
    dy = to_dev(y)
    qs.sort_segmented(dy, to_dev(np.array([0, y.size], dtype=np.int64)))
    torch.cuda.synchronize()
    assert_keys_equal(dy.cpu().numpy(), oracle.sort(y))
    # no segments: nothing happens
    z = to_dev(synth.uniform_i32(100, 48))
    before = z.clone()
    qs.sort_segmented(z, torch.zeros(1, dtype=torch.int64, device="cuda"))
    assert bool((z == before).all())


def test_segmented_rejects_bad_offsets():
    import torch

    qs = qs_gpu()
    d = to_dev(synth.uniform_i32(1000, 49))
    with pytest.raises(qs.QSError) as e:
        qs.sort_segmented(d, to_dev(np.array([0, 600, 400, 1000], dtype=np.int64)))
    assert e.value.code == -1
    with pytest.raises(qs.QSError):
        qs.sort_segmented(d, to_dev(np.array([0, 500, 1001], dtype=np.int64)))
    # the library stays usable
    x = synth.uniform_i32(1000, 50)
    d = to_dev(x)
    qs.sort_segmented(d, to_dev(np.array([0, 500, 1000], dtype=np.int64)))
    torch.cuda.synchronize()
    _check_segments(x, d.cpu().numpy(), np.array([0, 500, 1000]))


def test_segmented_graph_replay_new_data():
    """Same buffers and offsets twice (the cached graph is replayed) with new data."""
    import torch

    qs = qs_gpu()
    offs = _segments(120, 51, hi=1 << 15)
    n = int(offs[-1])
    d = torch.empty(n, dtype=torch.int32, device="cuda")
    doffs = to_dev(offs)
    for seed in (52, 53, 54):
        x = synth.uniform_i32(n, seed)
        d.copy_(torch.from_numpy(x))
        qs.sort_segmented(d, doffs)
        torch.cuda.synchronize()
        _check_segments(x, d.cpu().numpy(), offs)


def test_segmented_full_workload():
    """20,000 int32 segments, sizes log-uniform in [16, 2^18] (~540 M keys): every
    segment sorted and a permutation of its input (checked on the GPU), plus 40
    sampled segments against the oracle."""
    import torch

    qs = qs_gpu()
    keys, offs = synth.segments_i32(20_000)
    n = keys.size
    d = torch.from_numpy(keys).to("cuda")
    doffs = torch.from_numpy(offs).to("cuda")
    seg_id = torch.repeat_interleave(torch.arange(20_000, device="cuda"), doffs[1:] - doffs[:-1])

    def seg_hash(t):
        z = t.to(torch.int64) * 0x1F3D5B79 + seg_id * 0x5851F42D
        z = z ^ (z >> 29)
        return torch.zeros(20_000, dtype=torch.int64, device="cuda").index_add_(0, seg_id, z)

    h_in = seg_hash(d)
    qs.sort_segmented(d, doffs)
    torch.cuda.synchronize()
    ok_order = (d[1:] >= d[:-1]) | (seg_id[1:] != seg_id[:-1])
    assert bool(ok_order.all()), "a segment is not sorted"
    assert bool((seg_hash(d) == h_in).all()), "a segment is not a permutation of its input"
    got = d.cpu().numpy()
    rng = np.random.default_rng(55)
    _check_segments(keys, got, offs, segs=[int(i) for i in rng.integers(0, 20_000, 40)])


def test_segmented_full_workload_kv():
    """The key/value variant of the 20,000-segment workload (values = original
    index): on the GPU, every segment's keys are sorted, every output value
    points back to an input position of the same segment holding the same key,
    and the values are a permutation; plus 40 sampled segments against the
    oracle (keys bit-exact, equal-key runs as value multisets)."""
    import torch

    qs = qs_gpu()
    keys, offs = synth.segments_i32(20_000)
    n = keys.size
    vals = np.arange(n, dtype=np.int32)
    dk = torch.from_numpy(keys).to("cuda")
    dv = torch.from_numpy(vals).to("cuda")
    keys_in = dk.clone()
    doffs = torch.from_numpy(offs).to("cuda")
    seg_id = torch.repeat_interleave(torch.arange(20_000, device="cuda", dtype=torch.int32),
                                     doffs[1:] - doffs[:-1])
    qs.sort_segmented(dk, doffs, dv)
    torch.cuda.synchronize()
    assert bool(((dk[1:] >= dk[:-1]) | (seg_id[1:] != seg_id[:-1])).all()), "a segment's keys are not sorted"
    v64 = dv.to(torch.int64)
    assert bool(((v64 >= 0) & (v64 < n)).all())
    assert bool((keys_in[v64] == dk).all()), "a value does not point at its key"
    assert bool((seg_id[v64] == seg_id).all()), "a value left its segment"
    seen = torch.zeros(n, dtype=torch.int32, device="cuda").index_add_(0, v64, torch.ones_like(dv))
    assert bool((seen == 1).all()), "values are not a permutation"
    del seen, v64, keys_in, seg_id
    gk, gv = dk.cpu().numpy(), dv.cpu().numpy()
    rng = np.random.default_rng(56)
    _check_segments(keys, gk, offs, segs=[int(i) for i in rng.integers(0, 20_000, 40)], vals_in=vals, vals_out=gv)


@pytest.mark.parametrize("kind", ["i32", "kv"])
def test_autotune_applies_caches_and_sorts_right(kind, tmp_path, monkeypatch):
    """paper_1704_08579_gb300.autotune: the chosen leaf threshold, one-warp
    threshold and tile variant come from the candidate lists, are applied
    (read back with qs_get_option), are stored in the cache and returned from
    it on the next call, and the segmented sort under them matches the oracle
    per segment."""
    import torch

    from paper_1704_08579_gb300 import autotune

    qs = qs_gpu()
    monkeypatch.setattr(autotune, "CACHE_DIR", str(tmp_path))
    offs = _segments(250, 57, hi=1 << 16)
    n = int(offs[-1])
    x = synth.uniform_i32(n, 58)
    v = np.arange(n, dtype=np.int32) if kind == "kv" else None
    dk, doffs = to_dev(x), to_dev(offs)
    dv = to_dev(v) if v is not None else None
    try:
        res = autotune.tune(dk, doffs, dv, reps=1, use_cache=True)
        assert res["leaf_max"] in autotune.LEAF_CHOICES[kind]
        assert res["small_max"] in autotune.SMALL_CHOICES and res["small_max"] <= res["leaf_max"]
        assert res["driver_items"] in autotune.ITEMS_CHOICES[kind]
        assert len(res["table"]) >= 2 and res["ms"] == min(r["ms"] for r in res["table"])
        for name in ("leaf_max", "small_max", "driver_items"):
            assert qs.get_option(name) == res[name]
        np.testing.assert_array_equal(dk.cpu().numpy(), x)  # tuning leaves the input alone
        autotune.apply({})
        again = autotune.tune(dk, doffs, dv, reps=1, use_cache=True)
        assert again.get("cached") is True
        for name in ("leaf_max", "small_max", "driver_items"):
            assert again[name] == res[name] and qs.get_option(name) == res[name]
        qs.sort_segmented(dk, doffs, dv)
        torch.cuda.synchronize()
        if v is None:
            _check_segments(x, dk.cpu().numpy(), offs)
        else:
            _check_segments(x, dk.cpu().numpy(), offs, vals_in=v, vals_out=dv.cpu().numpy())
    finally:
        autotune.apply({})
