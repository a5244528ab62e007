"""GPU parity of the leaf kernel's mid-range stage against the oracle.

With QS_OPT_LEAF_MAX above LEAF (what one CTA's shared memory sorts: 16384
f64 or key/value pairs, 32768 int32), up to MID = 2 * LEAF, a part of more
than LEAF keys is not split by one more device-wide partition pass: the leaf
kernel's CTA picks a sampled pivot and partitions it once itself (Section
III-B's two write cursors, one chunk at a time), then sorts the sides.
Covered here: every size class around LEAF and MID, arrays that are one
mid-range part, the equal-key rules inside the split ('<' moving nothing,
then '<='; a side of only pivot-equal keys; a side still above LEAF that
needs a second split), pinned host buffers (sides written to a separate
output), segmented sorts with segments in (LEAF, MID], and the default
threshold, which leaves the stage off.  Keys bit-exact; key/value pairs:
value multisets per equal-key run and every pair intact.
"""
import numpy as np
import pytest

import oracle
import synth
from qs_testutil import assert_keys_equal, assert_kv_sorted_equal, oracle_sort, qs_gpu, to_dev

pytestmark = pytest.mark.gpu

LEAF = {"i32": 32768, "f64": 16384, "kv": 16384}


@pytest.fixture
def mid_on(request):
    """Leaf threshold at MID for the test's kind (restored afterwards)."""
    qs = qs_gpu()
    qs.set_option("leaf_max", 2 * LEAF[request.node.callspec.params["kind"]])
    yield qs
    qs.set_option("leaf_max", 0)


def _keys(kind, n, seed):
    if kind == "i32":
        return synth.uniform_i32(n, seed), None
    if kind == "f64":
        return synth.uniform_f64(n, seed), None
    return synth.mod_i32(n, seed, 1 << 20), np.arange(n, dtype=np.int32)


def _sort(qs, k, v=None):
    import torch

    dk = to_dev(k)
    dv = to_dev(v) if v is not None else None
    qs.sort(dk, dv)
    torch.cuda.synchronize()
    return dk.cpu().numpy(), (dv.cpu().numpy() if v is not None else None)


def _check(k, v, gk, gv):
    if v is None:
        assert_keys_equal(gk, oracle_sort(k))
    else:
        ok, ov = oracle_sort(k, v)
        assert_kv_sorted_equal(k, v, gk, gv, ok, ov)
        np.testing.assert_array_equal(k[gv], gk)  # value = original index: pairs intact


@pytest.mark.parametrize("kind", ["i32", "f64", "kv"])
def test_mid_sizes(kind, mid_on):
    """Sizes at and around LEAF and MID; an array of LEAF < n <= MID keys is
    one mid-range part (one split, counted in qs_stats)."""
    qs = mid_on
    L = LEAF[kind]
    for n in (L + 1, L + 777, 2 * L - 1, 2 * L, 2 * L + 1, 3 * L + 5, 8 * L + 3):
        k, v = _keys(kind, n, 700 + n)
        gk, gv = _sort(qs, k, v)
        _check(k, v, gk, gv)
        st = qs.stats()
        if n <= 2 * L:
            assert st["part_tasks"] == 0 and st["mid_parts"] >= 1 and st["mid_keys"] >= n


def _dup_cases(kind, n):
    """Inputs that drive the split's equal-key rules."""
    rng = np.random.default_rng(n)
    base = rng.integers(-1000, 1000, n)
    cases = {
        "all_equal": np.full(n, 5),
        "two_valued": np.where(rng.integers(0, 2, n) == 0, -3, 9),
        # 60 % one value in the middle: the pivot is that value, the upper side
        # (>= pivot) stays above LEAF and is split again ('<' moves nothing,
        # then '<=' finishes the equal run).
        "heavy_median": np.where(rng.integers(0, 10, n) < 6, 0, base),
        # 90 % the smallest value: the pivot is the minimum ('<=' pass first).
        "heavy_min": np.where(rng.integers(0, 10, n) < 9, -5000, base),
        # 90 % the largest value: the upper side holds only pivot-equal keys.
        "heavy_max": np.where(rng.integers(0, 10, n) < 9, 5000, base),
    }
    out = {}
    for name, c in cases.items():
        if kind == "f64":
            out[name] = (c.astype(np.float64) * 0.25, None)
        elif kind == "i32":
            out[name] = (c.astype(np.int32), None)
        else:
            out[name] = (c.astype(np.int32), np.arange(n, dtype=np.int32))
    return out


@pytest.mark.parametrize("kind", ["i32", "f64", "kv"])
def test_mid_equal_keys(kind, mid_on):
    qs = mid_on
    L = LEAF[kind]
    for n in (L + 1, 2 * L - 3, 2 * L):
        for name, (k, v) in _dup_cases(kind, n).items():
            gk, gv = _sort(qs, k, v)
            _check(k, v, gk, gv)


@pytest.mark.parametrize("kind", ["i32", "f64", "kv"])
def test_mid_skewed_values(kind, mid_on):
    """Log-normal keys: the sides of a split are unequal, some above LEAF."""
    qs = mid_on
    L = LEAF[kind]
    for n in (2 * L, 5 * L + 11):
        x = synth.lognormal_f64(n, 900 + n)
        if kind == "f64":
            k, v = x, None
        else:
            k = np.clip(x * 1e4, -2**31, 2**31 - 1).astype(np.int32)
            v = np.arange(n, dtype=np.int32) if kind == "kv" else None
        gk, gv = _sort(qs, k, v)
        _check(k, v, gk, gv)


def _pinned(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()


@pytest.mark.parametrize("kind", ["i32", "f64", "kv"])
def test_mid_pinned_host_buffers(kind, mid_on):
    """Sorted sides and finished equal runs go straight to a separate output
    (mapped pinned host memory), also when they were split in place."""
    qs = mid_on
    L = LEAF[kind]
    for n in (2 * L, 3 * L + 1):
        cases = [_keys(kind, n, 60 + n)] + list(_dup_cases(kind, n).values())
        for k, v in cases:
            hk = _pinned(k)
            hv = _pinned(v) if v is not None else None
            qs.sort_host(hk, hv)
            _check(k, v, hk, hv)


@pytest.mark.parametrize("kind", ["i32", "f64", "kv"])
def test_mid_segmented(kind, mid_on):
    """Segments of every size class, many of them in (LEAF, MID]."""
    import torch

    qs = mid_on
    L = LEAF[kind]
    rng = np.random.default_rng(77)
    sizes = np.concatenate([rng.integers(L + 1, 2 * L + 1, 24), rng.integers(1, 3 * L, 24), [0, 1, 2 * L, L]])
    rng.shuffle(sizes)
    offs = np.zeros(sizes.size + 1, np.int64)
    np.cumsum(sizes, out=offs[1:])
    n = int(offs[-1])
    k, v = _keys(kind, n, 81)
    dk = to_dev(k)
    dv = to_dev(v) if v is not None else None
    qs.sort_segmented(dk, to_dev(offs), dv)
    torch.cuda.synchronize()
    gk = dk.cpu().numpy()
    gv = dv.cpu().numpy() if v is not None else None
    assert qs.stats()["mid_parts"] >= 24
    for i in range(sizes.size):
        a, b = int(offs[i]), int(offs[i + 1])
        if v is None:
            assert_keys_equal(gk[a:b], oracle.sort(k[a:b]))
        else:
            ok, ov = oracle.sort(k[a:b], v[a:b])
            assert_kv_sorted_equal(k[a:b], v[a:b], gk[a:b], gv[a:b], ok, ov)


@pytest.mark.parametrize("kind", ["i32", "f64", "kv"])
def test_mid_stage_default_off(kind):
    """The default leaf threshold (QS_OPT_LEAF_MAX = 0) is LEAF: no part above
    it reaches the leaf kernel and no split runs there; at MID splits run.
    Both give the oracle's result."""
    qs = qs_gpu()
    L = LEAF[kind]
    n = 6 * L + 5
    k, v = _keys(kind, n, 99)
    gk, gv = _sort(qs, k, v)
    assert qs.stats()["mid_parts"] == 0
    _check(k, v, gk, gv)
    try:
        qs.set_option("leaf_max", 2 * L)
        gk2, gv2 = _sort(qs, k, v)
        assert qs.stats()["mid_parts"] > 0
        _check(k, v, gk2, gv2)
        qs.set_option("leaf_max", 4 * L)  # clamped to MID
        gk3, gv3 = _sort(qs, k, v)
        _check(k, v, gk3, gv3)
    finally:
        qs.set_option("leaf_max", 0)
