"""Pins for the reading of the paper's Bitonic network (Section III-A).

Algorithm 1 prints its network as six permutation-and-blend stages on one
vector of 8 lanes (``tests/golden/alg1_bitonic8.txt``).  The leaf kernel runs
the same network by rule instead of by table: for every block size s = 2, 4,
..., P, element i meets its mirror i ^ (s - 1) inside the block (the "flip"
of Figure 2), then i ^ j for j = s/4, ..., 1; every comparator keeps the
minimum at the lower index.  These CPU tests check that reading against what
the paper and the mathematics fix:

  * the printed stages, applied with the intrinsics' meaning (lane i of the
    permuted vector is lane idx[i] of the input; the blend mask picks the
    maximum where its bit is set), sort every permutation and every 0-1 input
    of 8 lanes;
  * each printed stage is exactly the rule's stage at P = 8 (partners xor 1,
    3, 1, 7, 2, 1; the higher lane of every pair keeps the maximum);
  * the rule is a sorting network for every P up to 16 by the 0-1 principle
    (all 2^P inputs) and sorts random inputs with many duplicates up to 4096;
  * padding the tail with the largest key (Section III-A-3) is safe: with a
    comparator that swaps only on a strict inequality, no pad ever moves,
    even when real keys equal the padding value.
A mistake in the decoding (reading the table lowest lane first, a swapped
min/max mask, the half-cleaners starting at s/2 after the flip) fails one of
them.
"""
import itertools
import os

import numpy as np
import pytest

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _paper_stages():
    """(lane permutation, max mask) per stage of Algorithm 1, lane 0 first."""
    stages = []
    with open(os.path.join(GOLDEN, "alg1_bitonic8.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            fields = line.split()
            assert fields[0] == "stage"
            printed = [int(v) for v in fields[2:10]]  # lane 7 first
            perm = np.array(printed[::-1])
            mask = int(fields[10], 16)
            stages.append((perm, mask))
    return stages


def _apply_paper_stage(x, perm, mask):
    """One stage with the intrinsics' meaning: permute, min, max, blend."""
    neigh = x[..., perm]
    mn = np.minimum(x, neigh)
    mx = np.maximum(x, neigh)
    takes_max = np.array([(mask >> i) & 1 for i in range(x.shape[-1])], dtype=bool)
    return np.where(takes_max, mx, mn)


def _rule_masks(p):
    """Partner masks of the flip-form network on p elements, in order."""
    masks = []
    s = 2
    while s <= p:
        masks.append(s - 1)
        j = s // 4
        while j >= 1:
            masks.append(j)
            j //= 2
        s *= 2
    return masks


def _apply_rule(x, ids=None):
    """The rule's network on the last axis; a pair swaps only when the upper
    element is strictly smaller.  ids (same shape) follow their keys."""
    p = x.shape[-1]
    idx = np.arange(p)
    x = x.copy()
    ids = None if ids is None else ids.copy()
    for m in _rule_masks(p):
        partner = idx ^ m
        lower = idx < partner
        lo_i, hi_i = idx[lower], partner[lower]
        a, b = x[..., lo_i], x[..., hi_i]
        sw = b < a
        x[..., lo_i], x[..., hi_i] = np.where(sw, b, a), np.where(sw, a, b)
        if ids is not None:
            ia, ib = ids[..., lo_i], ids[..., hi_i]
            ids[..., lo_i], ids[..., hi_i] = np.where(sw, ib, ia), np.where(sw, ia, ib)
    return x if ids is None else (x, ids)


def _all_01(p):
    return ((np.arange(1 << p)[:, None] >> np.arange(p)[None, :]) & 1).astype(np.int64)


def test_paper_stages_sort_every_permutation_and_01_input():
    stages = _paper_stages()
    assert len(stages) == 6
    for inputs in (np.array(list(itertools.permutations(range(8)))), _all_01(8)):
        x = inputs.astype(np.float64)
        for perm, mask in stages:
            x = _apply_paper_stage(x, perm, mask)
        assert np.array_equal(x, np.sort(inputs, axis=1))


def test_paper_stages_are_the_flip_rule():
    stages = _paper_stages()
    masks = _rule_masks(8)
    assert masks == [1, 3, 1, 7, 2, 1]
    lanes = np.arange(8)
    for (perm, mask), m in zip(stages, masks):
        assert np.array_equal(perm, lanes ^ m)
        # the higher lane of each pair keeps the maximum
        assert all(((mask >> i) & 1) == (i > (i ^ m)) for i in range(8))


@pytest.mark.parametrize("p", [2, 4, 8, 16])
def test_rule_sorts_every_01_input(p):
    x = _all_01(p)
    assert np.array_equal(_apply_rule(x), np.sort(x, axis=1))


@pytest.mark.parametrize("p", [32, 256, 4096])
def test_rule_sorts_random_inputs_with_duplicates(p):
    rng = np.random.default_rng(p)
    for hi in (3, 50, 1 << 40):
        x = rng.integers(0, hi, size=(8, p), dtype=np.int64)
        assert np.array_equal(_apply_rule(x), np.sort(x, axis=1))


@pytest.mark.parametrize("n", [1, 17, 33, 63])
def test_padding_with_the_largest_key_never_moves(n):
    p = 64
    top = np.iinfo(np.int64).max
    rng = np.random.default_rng(n)
    x = np.full((16, p), top, dtype=np.int64)
    real = rng.integers(0, 5, size=(16, n), dtype=np.int64)
    real[:, ::3] = top  # real keys equal to the padding value
    x[:, :n] = real
    ids = np.broadcast_to(np.arange(p), (16, p)).copy()
    y, yid = _apply_rule(x, ids)
    assert np.array_equal(yid[:, n:], ids[:, n:])  # every pad where it started
    assert np.array_equal(y[:, :n], np.sort(real, axis=1))
