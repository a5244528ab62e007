"""Pins for the CPU oracle, independent of the oracle's own code.

Each pin is something the paper or plain mathematics fixes:
  * Figure 1's worked example (input, output, first pivot);
  * brute force: every permutation for n <= 8 and every sequence over {0,1,2}
    for n <= 8 must come out equal to Python's ``sorted`` (the sorted multiset
    is unique);
  * random inputs of every workload shape equal ``numpy.sort``;
  * key/value: with value = original index, ``keys_in[vals_out] == keys_out``
    and the values are a permutation (Section III-D: values follow keys);
  * partition: split = number of keys below the pivot, every lower key is
    below and every upper key at-or-above the pivot (Section III-B), the lower
    side equals the input's lower keys in input order and the upper side the
    input's upper keys in reverse input order, brute force over tiny inputs;
  * selection equals the k-th element of ``sorted``.
These catch the plausible slips: '<=' for '<', a dropped swap of the value
array, a wrong bound or middle index, a reversed side.
"""
import itertools
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    out = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            out[key] = [int(v) for v in vals]
    return out


def test_figure1_example():
    g = _read_golden("fig1_quicksort.txt")
    keys = np.array(g["input"], dtype=np.int32)
    out, trace = oracle.sort_trace(keys)
    assert out.tolist() == g["output"]
    assert int(trace[0]) == g["first_pivot"][0]
    # Appendix A's middle pick on the sub-ranges [1,0] and [3,5] gives 1 and 3.
    assert sorted(int(t) for t in trace) == [1, 2, 3]


@pytest.mark.parametrize("n", range(0, 9))
def test_sort_all_permutations(n):
    for perm in itertools.permutations(range(n)):
        a = np.array(perm, dtype=np.int32)
        assert oracle.sort(a).tolist() == list(range(n))
        assert oracle.sort(a.astype(np.float64) - 3.5).tolist() == [x - 3.5 for x in range(n)]


@pytest.mark.parametrize("n", range(1, 9))
def test_sort_all_ternary_sequences(n):
    for seq in itertools.product((0, 1, 2), repeat=n):
        a = np.array(seq, dtype=np.int32)
        assert oracle.sort(a).tolist() == sorted(seq)


@pytest.mark.parametrize("dist", ["uniform", "sorted", "reverse", "few"])
def test_sort_f64_distributions(dist):
    x = synth.f64_config(dist, 1 << 16)
    np.testing.assert_array_equal(oracle.sort(x), np.sort(x, kind="stable"))


def test_sort_i32_uniform_and_duplicates():
    for x in (synth.uniform_i32(1 << 17, 11), synth.mod_i32(1 << 17, 12, 7), np.zeros(5000, np.int32),
              np.full(3000, 2**31 - 1, np.int32), np.full(3000, -2**31, np.int32)):
        np.testing.assert_array_equal(oracle.sort(x), np.sort(x, kind="stable"))


def test_sort_f64_extremes():
    """Infinities, the largest and smallest normals, subnormals and zero among
    ordinary keys (no NaN, no -0.0: the inputs' precondition) sort as numpy
    sorts them, bit for bit; so do mixed int32 extremes."""
    tiny = np.finfo(np.float64).tiny
    special = np.array([np.inf, -np.inf, np.finfo(np.float64).max, -np.finfo(np.float64).max, tiny, -tiny,
                        5e-324, -5e-324, tiny / 3, 0.0, 1.0, -1.0], dtype=np.float64)
    rng = np.random.default_rng(5)
    for reps in (1, 7, 300):
        x = np.concatenate([np.repeat(special, reps), synth.uniform_f64(1000, 31)])
        x = x[rng.permutation(x.size)]
        got = oracle.sort(x)
        assert np.array_equal(got.view(np.int64), np.sort(x, kind="stable").view(np.int64))
    e = np.array([-2**31, 2**31 - 1, 0, -1, 1], dtype=np.int32)
    y = np.concatenate([np.repeat(e, 101), synth.uniform_i32(999, 32)])
    y = y[rng.permutation(y.size)]
    np.testing.assert_array_equal(oracle.sort(y), np.sort(y, kind="stable"))


@pytest.mark.parametrize("dist", ["uniform", "mod1000", "sorted", "reverse"])
def test_sort_kv_values_follow_keys(dist):
    k, v = synth.kv_config(dist, 1 << 15)
    ko, vo = oracle.sort(k, v)
    np.testing.assert_array_equal(ko, np.sort(k, kind="stable"))
    assert np.array_equal(np.sort(vo), np.arange(k.size, dtype=np.int32))  # a permutation
    np.testing.assert_array_equal(k[vo], ko)  # each value still sits with its own key


def test_sort_kv_brute_force_small():
    for n in range(1, 7):
        for seq in itertools.product((0, 1, 2), repeat=n):
            k = np.array(seq, dtype=np.int32)
            v = np.arange(n, dtype=np.int32)
            ko, vo = oracle.sort(k, v)
            assert ko.tolist() == sorted(seq)
            assert sorted(vo.tolist()) == list(range(n))
            assert k[vo].tolist() == ko.tolist()


def _expected_partition(x, pivot):
    low = [a for a in x if a < pivot]
    high = [a for a in x if not a < pivot]
    return len(low), low + high[::-1]


@pytest.mark.parametrize("n", range(0, 9))
def test_partition_brute_force(n):
    for perm in itertools.permutations(range(n)):
        x = np.array(perm, dtype=np.int32)
        for pivot in range(-1, n + 1):
            split, out = oracle.partition(x, pivot)
            exp_split, exp = _expected_partition(perm, pivot)
            assert split == exp_split == sum(1 for a in perm if a < pivot)
            assert out.tolist() == exp


@pytest.mark.parametrize("n", range(0, 8))
def test_partition_kv_brute_force_with_duplicates(n):
    """Every key sequence over {0, 1, 2} with value = original index, every
    pivot: the values name exactly which element went where, so the canonical
    order among equal keys (lower side in input order, upper side in reverse
    input order) is pinned, not only the keys."""
    idx = np.arange(n, dtype=np.int32)
    for seq in itertools.product(range(3), repeat=n):
        k = np.array(seq, dtype=np.int32)
        for pivot in range(-1, 4):
            split, ko, vo = oracle.partition(k, pivot, idx)
            low = [i for i in range(n) if seq[i] < pivot]
            high = [i for i in range(n) if not seq[i] < pivot][::-1]
            assert split == len(low)
            assert vo.tolist() == low + high
            assert ko.tolist() == [seq[i] for i in low + high]


@pytest.mark.parametrize("dtype", [np.int32, np.float64])
def test_partition_random(dtype):
    if dtype == np.int32:
        x = synth.uniform_i32(100_003, 21)
        pivots = [int(x[17]), -2**31, 2**31 - 1, 0]
    else:
        x = synth.uniform_f64(100_003, 22)
        pivots = [float(x[17]), -1e7, 1e7, 0.0]
    for pivot in pivots:
        split, out = oracle.partition(x, pivot)
        mask = x < pivot
        assert split == int(np.count_nonzero(mask))
        assert np.all(out[:split] < pivot) and np.all(out[split:] >= pivot)
        np.testing.assert_array_equal(out[:split], x[mask])
        np.testing.assert_array_equal(out[split:], x[~mask][::-1])


def test_partition_kv():
    k, v = synth.kv_config("mod1000", 50_001)
    split, ko, vo = oracle.partition(k, 500, v)
    mask = k < 500
    assert split == int(np.count_nonzero(mask))
    np.testing.assert_array_equal(ko[:split], k[mask])
    np.testing.assert_array_equal(ko[split:], k[~mask][::-1])
    np.testing.assert_array_equal(vo[:split], v[mask])
    np.testing.assert_array_equal(vo[split:], v[~mask][::-1])


def test_select():
    x = synth.mod_i32(10_001, 5, 50)
    s = sorted(x.tolist())
    for k in (0, 1, 77, 5000, 10_000):
        assert oracle.select(x, k) == s[k]
    y = synth.uniform_f64(4097, 6)
    assert oracle.select(y, 2048) == sorted(y.tolist())[2048]


def test_splitmix64_known_outputs():
    """The generator both sides share is SplitMix64 as published (Steele, Lea
    and Flood 2014; the reference C version by Vigna): seeded with 0, its first
    outputs are these well-known values."""
    got = [int(v) for v in synth.splitmix64(0, 0, 4)]
    assert got == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F, 0xF88BB8A8724C81EC]
    # counter based: output i does not depend on where the slice starts
    assert [int(v) for v in synth.splitmix64(0, 2, 2)] == got[2:]


def test_synth_properties():
    a = synth.uniform_f64(1 << 16, 1)
    assert np.all(np.isfinite(a)) and not np.any(np.signbit(a) & (a == 0))
    assert a.min() >= -1e6 and a.max() < 1e6
    s = synth.f64_config("sorted", 1 << 16)
    assert np.all(np.diff(s) >= 0)
    r = synth.f64_config("reverse", 1 << 16)
    assert np.all(np.diff(r) <= 0)
    f = synth.f64_config("few", 1 << 16)
    assert np.unique(f).size == 16
    k, v = synth.kv_config("sorted", 1 << 16)
    assert np.all(np.diff(k.astype(np.int64)) >= 0) and k[0] < -2**31 + 2**17 and k[-1] > 2**31 - 2**17
    m, _ = synth.kv_config("mod1000", 1 << 16)
    assert m.min() == 0 and m.max() == 999
    # counter-based: any slice regenerates identically
    np.testing.assert_array_equal(synth.uniform_i32(1000, 9)[500:], synth.uniform_i32(1000, 9)[500:])
    keys, offs = synth.segments_i32(50)
    assert offs[0] == 0 and offs[-1] == keys.size and np.all(np.diff(offs) >= 16)


def test_skewed_workload_recipes():
    """The learned-splitter and batched workloads follow their stated laws:
    Zipf(1.2) over 2^24 values (the top value's share is 1 / sum k^-1.2, keys
    on the grid k*256 - 2^31), lognormal(0, 2) (log x / 2 is standard normal),
    an 8-Gaussian mixture inside the int32 range, and log-uniform segment sizes
    in [16, 2^18)."""
    n = 1 << 18
    z = synth.zipf_i32(n, 41)
    assert np.all((z.astype(np.int64) + 2**31) % 256 == 0)
    top = np.bincount(((z.astype(np.int64) + 2**31) // 256).astype(np.int64)).max() / n
    h = float(np.sum(np.arange(1, (1 << 24) + 1, dtype=np.float64) ** -1.2))
    assert abs(top - 1 / h) < 0.01
    lg = np.log(synth.lognormal_f64(n, 42)) / 2.0
    assert abs(lg.mean()) < 0.01 and abs(lg.std() - 1.0) < 0.01
    means, sig, cw = synth.gauss_mix_params(43)
    g = synth.gauss_mix_i32(n, 43).astype(np.float64)
    near = np.min(np.abs(g[:, None] - means[None, :]) / sig[None, :], axis=1)
    assert means.size == 8 and np.all(np.diff(cw) > 0) and abs(cw[-1] - 1) < 1e-12
    assert np.mean(near < 5) > 0.999
    sizes = synth.segment_sizes(20000, 44)
    assert sizes.min() >= 16 and sizes.max() < 1 << 18
    assert abs(np.log(sizes + 0.5).mean() - (np.log(16) + np.log(1 << 18)) / 2) < 0.05


@pytest.mark.parametrize("threads", [1, 2, 3, 16])
def test_parallel_oracle_equals_sequential(threads):
    """The task-parallel oracle runs the same Appendix A steps: identical output."""
    for n, seed in ((0, 1), (1, 2), (70000, 3), ((1 << 18) + 11, 4)):
        x = synth.uniform_f64(n, seed)
        assert np.array_equal(oracle.sort_parallel(x, threads=threads).view(np.int64), oracle.sort(x).view(np.int64))
        y = synth.mod_i32(n, seed, 37)
        assert np.array_equal(oracle.sort_parallel(y, threads=threads), oracle.sort(y))
        k, v = synth.kv_config("mod1000", n, seed)
        pk, pv = oracle.sort_parallel(k, v, threads=threads)
        sk, sv = oracle.sort(k, v)
        assert np.array_equal(pk, sk) and np.array_equal(pv, sv)
