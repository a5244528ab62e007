"""qs_partition_i32_noalloc, the entry point for callers that may not allocate
device memory (its scratch is a fixed device array instead of the growable
workspace).  It must give exactly what qs_partition_i32 gives.  This file is
collected last so that a run stopping at the first failure has already run
every other test."""
import ctypes

import numpy as np
import pytest

import synth
from qs_testutil import qs_gpu, to_dev

pytestmark = pytest.mark.gpu

MAX_N = 1 << 20  # QS_NOALLOC_MAX_N in include/qs.h


def test_noalloc_partition_matches_regular_entry_point():
    import torch

    qs = qs_gpu()
    lib = qs.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    # Two calls in a row (the shared scratch keeps the previous call's contents).
    for call, n in enumerate((MAX_N, 100_003)):
        x = synth.uniform_i32(n, 900 + call)
        pivot = int(x[n // 3])
        ref = to_dev(x)
        got = to_dev(x)
        split_ref = lib.qs_partition_i32(ctypes.c_void_p(ref.data_ptr()), n, pivot, stream)
        split_got = lib.qs_partition_i32_noalloc(ctypes.c_void_p(got.data_ptr()), n, pivot, stream)
        torch.cuda.synchronize()
        assert split_ref >= 0 and split_got == split_ref
        np.testing.assert_array_equal(got.cpu().numpy(), ref.cpu().numpy())


def test_noalloc_rejects_sizes_beyond_its_maximum():
    import torch

    qs = qs_gpu()
    lib = qs.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    buf = torch.zeros(8, dtype=torch.int32, device="cuda")
    assert lib.qs_partition_i32_noalloc(ctypes.c_void_p(buf.data_ptr()), MAX_N + 1, 0, stream) == -1
    assert lib.qs_partition_i32_noalloc(ctypes.c_void_p(buf.data_ptr()), 0, 0, stream) == 0
