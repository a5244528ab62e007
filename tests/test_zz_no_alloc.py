"""qs_partition_i32_noalloc, the partition for callers that cannot let the
library allocate device memory: code that works inside a fixed device-memory
budget handed out by its own allocator, or that must never be stalled by the
device-wide synchronisation of cudaFree with which the regular workspace is
resized.  Its scratch is one fixed device array instead of the growable
workspace.  Its split index and every output element must
equal the oracle's partition (Section III-B, with the lower side in input
order and the upper side in reverse input order), exactly as
qs_partition_i32's do.  This file is collected last so that a run stopping at
the first failure has already run every other test."""
import ctypes

import numpy as np
import pytest

import synth
from qs_testutil import assert_keys_equal, oracle_partition, qs_gpu, to_dev

pytestmark = pytest.mark.gpu

MAX_N = 1 << 20  # QS_NOALLOC_MAX_N in include/qs.h


def _noalloc(lib, x, pivot, stream, koff=0):
    """Runs the entry point on a device copy of x that starts koff int32
    elements into its allocation (koff = 1: 4 bytes past 16-byte alignment)."""
    import torch

    n = x.size
    buf = to_dev(np.concatenate([np.zeros(koff, np.int32), x]))
    d = buf[koff:koff + n]
    split = lib.qs_partition_i32_noalloc(ctypes.c_void_p(d.data_ptr()), n, int(pivot), stream)
    torch.cuda.synchronize()
    return split, d.cpu().numpy()


def _stream():
    import torch

    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def test_noalloc_partition_matches_oracle_two_calls_in_a_row():
    """The largest size, then a ragged one: the second call runs on scratch
    that still holds the first call's contents."""
    qs = qs_gpu()
    lib = qs.load()
    for call, n in enumerate((MAX_N, 100_003)):
        x = synth.uniform_i32(n, 900 + call)
        pivot = x[n // 3]
        split, got = _noalloc(lib, x, pivot, _stream())
        exp_split, exp = oracle_partition(x, pivot)
        assert split == exp_split
        assert_keys_equal(got, exp)


@pytest.mark.parametrize("n", [1, 5000])
@pytest.mark.parametrize("where", ["inside", "below_min", "above_max"])
def test_noalloc_small_sizes_and_outside_pivots(n, where):
    """n = 1 and a size below one partition tile; pivots inside the key range,
    below its minimum (split 0) and above its maximum (split n)."""
    qs = qs_gpu()
    lib = qs.load()
    x = synth.mod_i32(n, 910 + n, 1000) if n > 1 else np.array([17], dtype=np.int32)
    pivot = {"inside": x[n // 2], "below_min": x.min() - 1, "above_max": x.max() + 1}[where]
    split, got = _noalloc(lib, x, pivot, _stream())
    exp_split, exp = oracle_partition(x, np.int32(pivot))
    assert split == exp_split
    assert split == {"inside": exp_split, "below_min": 0, "above_max": n}[where]
    assert_keys_equal(got, exp)


@pytest.mark.parametrize("koff", [1, 3])
def test_noalloc_unaligned_pointer(koff):
    """Keys starting 4 or 12 bytes past a 16-byte boundary take the unaligned
    head path of the partition tile."""
    qs = qs_gpu()
    lib = qs.load()
    x = synth.uniform_i32(3 * 4096 + 17, 920 + koff)
    pivot = x[7]
    split, got = _noalloc(lib, x, pivot, _stream(), koff=koff)
    exp_split, exp = oracle_partition(x, pivot)
    assert split == exp_split
    assert_keys_equal(got, exp)


def test_noalloc_agrees_with_regular_entry_point():
    """Two calls in a row, each against qs_partition_i32 on the same input:
    the same split and the same keys in the same order."""
    import torch

    qs = qs_gpu()
    lib = qs.load()
    for n, seed in ((250_001, 930), (MAX_N, 931)):
        x = synth.uniform_i32(n, seed)
        pivot = int(x[11])
        ref = to_dev(x)
        split_ref = lib.qs_partition_i32(ctypes.c_void_p(ref.data_ptr()), x.size, pivot, _stream())
        split, got = _noalloc(lib, x, pivot, _stream())
        torch.cuda.synchronize()
        assert split == split_ref
        assert_keys_equal(got, ref.cpu().numpy())


def test_noalloc_honours_the_wait_limit_and_recovers():
    """QS_OPT_WAIT_LIMIT_NS applies here as for qs_partition_i32: with a limit
    of 0 any wait of the persistent kernel (a tile's bulk copy, the
    look-back) that does not succeed at once ends the call with QS_ERR_TIMEOUT
    instead of hanging -- whether one happens depends on timing, so a call
    either reports the timeout or returns the right split -- and the next call
    with the normal limit is right again."""
    qs = qs_gpu()
    lib = qs.load()
    x = synth.uniform_i32(MAX_N, 940)
    pivot = x[5]
    exp_split, exp = oracle_partition(x, pivot)
    qs.set_option("wait_limit_ns", 0)
    try:
        results = [_noalloc(lib, x, pivot, _stream()) for _ in range(5)]
    finally:
        qs.set_option("wait_limit_ns", 2_000_000_000)
    for split, got in results:
        assert split in (-5, exp_split)
        if split == exp_split:
            assert_keys_equal(got, exp)
    split, got = _noalloc(lib, x, pivot, _stream())
    assert split == exp_split
    assert_keys_equal(got, exp)


def test_noalloc_rejects_sizes_beyond_its_maximum():
    import torch

    qs = qs_gpu()
    lib = qs.load()
    buf = torch.zeros(8, dtype=torch.int32, device="cuda")
    assert lib.qs_partition_i32_noalloc(ctypes.c_void_p(buf.data_ptr()), MAX_N + 1, 0, _stream()) == -1
    assert lib.qs_partition_i32_noalloc(ctypes.c_void_p(buf.data_ptr()), -1, 0, _stream()) == -1
    assert lib.qs_partition_i32_noalloc(ctypes.c_void_p(buf.data_ptr()), 0, 0, _stream()) == 0
    assert lib.qs_partition_i32_noalloc(ctypes.c_void_p(buf.data_ptr() + 2), 4, 0, _stream()) == -2
