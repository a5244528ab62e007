"""Parity at the benchmark's full sizes (n = 2^28): FP64 sorts of the four
distributions, qs_partition_f64 with the true median as pivot, and int32
key/value sorts of the four key distributions.

At this size the checks are:
  * the whole partition output against the oracle (a single O(n) pass);
  * for sorts, the whole key output against the oracle's sort (the
    task-parallel oracle, bit-for-bit the sequential one), plus properties
    that hold at any size: the output is non-decreasing and a permutation of
    the input (order-independent 64-bit hash of the multiset);
  * for key/value pairs with value = original index: every value appears once
    and keys_in[value_out] == keys_out (each pair is intact).
"""
import numpy as np
import pytest

import oracle
import synth
from qs_testutil import assert_keys_equal, qs_gpu

pytestmark = pytest.mark.gpu

N = 1 << 28


def _hash64(t):
    """Order-independent hash of a multiset of 64-bit words (SplitMix64 finaliser, summed mod 2^64)."""
    import torch

    z = t.view(torch.int64) if t.dtype == torch.float64 else t.to(torch.int64)
    z = z + 0x1E3779B97F4A7C15
    z = (z ^ (z >> 30)) * -4658895280553007687  # 0xBF58476D1CE4E5B9 as int64
    z = (z ^ (z >> 27)) * -7723592293110705685  # 0x94D049BB133111EB as int64
    z = z ^ (z >> 31)
    return int(z.sum().item())


def _check_sorted_permutation(dev_in_hash, out):
    import torch

    assert bool((out[1:] >= out[:-1]).all()), "output not sorted"
    assert _hash64(out) == dev_in_hash, "output is not a permutation of the input"


@pytest.mark.parametrize("dist", ["uniform", "sorted", "reverse", "few"])
def test_full_sort_f64(dist):
    import torch

    qs = qs_gpu()
    x = synth.f64_config(dist, N)
    d = torch.from_numpy(x).to("cuda")
    h_in = _hash64(d)
    qs.sort(d)
    torch.cuda.synchronize()
    _check_sorted_permutation(h_in, d)
    got = d.cpu().numpy()
    del d
    torch.cuda.empty_cache()
    assert_keys_equal(got, oracle.sort_parallel(x))


def test_full_partition_f64_true_median():
    import torch

    qs = qs_gpu()
    x = synth.f64_config("uniform", N)
    pivot = oracle.select(x, N // 2)  # the true (upper) median
    exp_split, exp = oracle.partition(x, pivot)
    d = torch.from_numpy(x).to("cuda")
    split = qs.partition(d, pivot)
    torch.cuda.synchronize()
    assert split == exp_split == N // 2
    assert_keys_equal(d.cpu().numpy(), exp)


@pytest.mark.parametrize("dist", ["uniform", "mod1000", "sorted", "reverse"])
def test_full_sort_kv(dist):
    import torch

    qs = qs_gpu()
    k, v = synth.kv_config(dist, N)
    dk = torch.from_numpy(k).to("cuda")
    dv = torch.from_numpy(v).to("cuda")
    keys_in = dk.clone()
    h_in = _hash64(dk)
    qs.sort(dk, dv)
    torch.cuda.synchronize()
    _check_sorted_permutation(h_in, dk)
    # value = original index: a permutation, and each value still sits with its own key
    counts = torch.bincount(dv.to(torch.int64), minlength=N)
    assert bool((counts == 1).all()), "values are not a permutation"
    assert bool((keys_in[dv.to(torch.int64)] == dk).all()), "a value was separated from its key"
    got = dk.cpu().numpy()
    del dk, dv, keys_in, counts
    torch.cuda.empty_cache()
    assert_keys_equal(got, oracle.sort_parallel(k))
