"""GPU parity of qs_partition_{i32,f64,kv} against the oracle (Section III-B).

The split index and every output element must match the oracle bit for bit:
the lower side in input order, the upper side in reverse input order.  Sizes
span several tiles (4096 keys for i32/kv, 2048 for f64) with ragged tails;
pointers are offset from 16-byte alignment to exercise the unaligned head.
"""
import numpy as np
import pytest

import synth
from qs_testutil import assert_keys_equal, oracle_partition, qs_gpu, to_dev

pytestmark = pytest.mark.gpu

SIZES = [1, 2, 3, 7, 100, 2047, 2048, 2049, 4095, 4096, 4097, 3 * 4096 + 17, 100_003, (1 << 20) + 5]


def _keys(kind, n, seed):
    if kind == "f64":
        return synth.uniform_f64(n, seed)
    return synth.uniform_i32(n, seed)


def _pivots(x):
    piv = [x[x.size // 2], x.min(), x.max()]
    if x.dtype == np.float64:
        piv += [x.max() + 1.0, x.min() - 1.0, 0.0]
    else:
        piv += [np.int32(2**31 - 1), np.int32(-2**31), np.int32(0)]
    return piv


def _run(qs, kind, x, pivot, v=None, koff=0, voff=0):
    import torch

    n = x.size
    kbuf = to_dev(np.concatenate([np.zeros(koff, x.dtype), x]))
    d = kbuf[koff:koff + n]
    if kind == "kv":
        vbuf = to_dev(np.concatenate([np.zeros(voff, np.int32), v]))
        dv = vbuf[voff:voff + n]
        split = qs.partition(d, pivot, dv)
        torch.cuda.synchronize()
        return split, d.cpu().numpy(), dv.cpu().numpy()
    split = qs.partition(d, pivot)
    torch.cuda.synchronize()
    return split, d.cpu().numpy()


@pytest.mark.parametrize("kind", ["i32", "f64"])
@pytest.mark.parametrize("n", SIZES)
def test_partition_keys(kind, n):
    qs = qs_gpu()
    x = _keys(kind, n, 1000 + n)
    for pivot in _pivots(x):
        exp_split, exp = oracle_partition(x, pivot)
        split, got = _run(qs, kind, x, pivot)
        assert split == exp_split, (pivot, split, exp_split)
        assert_keys_equal(got, exp)


@pytest.mark.parametrize("n", SIZES)
def test_partition_kv(n):
    qs = qs_gpu()
    k, v = synth.kv_config("mod1000", n, 77 + n)
    for pivot in (500, 0, 999, 1000, int(k[n // 2])):
        exp_split, ek, ev = oracle_partition(k, pivot, v)
        split, gk, gv = _run(qs, "kv", k, pivot, v)
        assert split == exp_split
        assert_keys_equal(gk, ek)
        np.testing.assert_array_equal(gv, ev)


@pytest.mark.parametrize("koff", [0, 1, 2, 3])
def test_partition_unaligned_i32(koff):
    qs = qs_gpu()
    n = 3 * 4096 + 9
    x = synth.uniform_i32(n, 5)
    exp_split, exp = oracle_partition(x, x[7])
    split, got = _run(qs, "i32", x, x[7], koff=koff)
    assert split == exp_split
    assert_keys_equal(got, exp)


def test_partition_unaligned_f64():
    qs = qs_gpu()
    n = 5 * 2048 + 3
    x = synth.uniform_f64(n, 6)
    exp_split, exp = oracle_partition(x, x[11])
    split, got = _run(qs, "f64", x, x[11], koff=1)
    assert split == exp_split
    assert_keys_equal(got, exp)


@pytest.mark.parametrize("koff,voff", [(0, 0), (1, 1), (1, 2), (0, 3), (3, 0)])
def test_partition_kv_phases(koff, voff):
    """Key and value arrays with different 16-byte phases."""
    qs = qs_gpu()
    n = 4 * 4096 + 13
    k, v = synth.kv_config("uniform", n, 8)
    exp_split, ek, ev = oracle_partition(k, int(k[3]), v)
    split, gk, gv = _run(qs, "kv", k, int(k[3]), v, koff, voff)
    assert split == exp_split
    assert_keys_equal(gk, ek)
    np.testing.assert_array_equal(gv, ev)


def test_partition_all_equal_and_empty():
    qs = qs_gpu()
    import torch

    x = np.full(10_001, 42, np.int32)
    for pivot in (41, 42, 43):
        exp_split, exp = oracle_partition(x, pivot)
        split, got = _run(qs, "i32", x, pivot)
        assert split == exp_split
        assert_keys_equal(got, exp)
    assert qs.partition(torch.zeros(0, dtype=torch.int32, device="cuda"), 3) == 0
