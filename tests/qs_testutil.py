"""Shared helpers for the GPU parity tests (comparison rules, device setup)."""
from __future__ import annotations

import numpy as np
import pytest

import oracle


def qs_gpu():
    """Builds (if needed) and loads the CUDA library; skips when no GPU is present."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1704_08579_gb300 import build as qs_build

    qs_build.build()
    import paper_1704_08579_gb300 as qs

    qs.load()
    return qs


def to_dev(a: np.ndarray):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda")


def assert_keys_equal(got: np.ndarray, exp: np.ndarray):
    """Bit-exact key comparison (FP64 compared by bit pattern)."""
    assert got.shape == exp.shape
    if got.dtype == np.float64:
        g, e = got.view(np.int64), exp.view(np.int64)
    else:
        g, e = got, exp
    if not np.array_equal(g, e):
        bad = np.flatnonzero(g != e)
        raise AssertionError("%d mismatches, first at %d: got %r expected %r"
                             % (bad.size, bad[0], got[bad[0]], exp[bad[0]]))


def assert_kv_sorted_equal(keys_in, vals_in, keys_out, vals_out, keys_oracle, vals_oracle):
    """Keys bit-exact vs the oracle; inside every run of equal keys the value
    multisets agree (the method is not stable, so the order of values among
    equal keys is free).  Also: each output pair exists in the input."""
    assert_keys_equal(keys_out, keys_oracle)
    n = keys_out.size
    if n == 0:
        return
    # Sort values inside each run of equal keys on both sides, then compare.
    run_id = np.concatenate(([0], np.cumsum(keys_oracle[1:] != keys_oracle[:-1])))
    order_g = np.lexsort((vals_out, run_id))
    order_o = np.lexsort((vals_oracle, run_id))
    np.testing.assert_array_equal(vals_out[order_g], vals_oracle[order_o])


def oracle_partition(keys, pivot, values=None):
    return oracle.partition(keys, pivot, values)


def oracle_sort(keys, values=None):
    return oracle.sort(keys, values)
