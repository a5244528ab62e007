"""Learned-splitter form at the benchmark's full sizes: 2^30 int32 keys
(Zipf(1.2) over 2^24 values; 8-Gaussian mixture) and 2^28 FP64 keys
(lognormal(0, 2)), generated on the device with the same recipes and
SplitMix64 streams as the host generators.

At this size the checks are: the whole output against the oracle's sort (the
task-parallel oracle, bit-for-bit the sequential one), bit-for-bit the output
of the plain sort of the same input, non-decreasing and a permutation of the
input (order-independent 64-bit hash of the multiset).  Sampled splitters, a model trained briefly with
the library's kernels and a deliberately bad model (one bucket takes almost
everything, so the size bound sends it to the plain method) are covered.
"""
import pytest

import oracle
from qs_testutil import assert_keys_equal, qs_gpu

pytestmark = pytest.mark.gpu


def _hash64(t):
    import torch

    z = t.view(torch.int64) if t.dtype == torch.float64 else t.to(torch.int64)
    z = z + 0x1E3779B97F4A7C15
    z = (z ^ (z >> 30)) * -4658895280553007687  # 0xBF58476D1CE4E5B9 as int64
    z = (z ^ (z >> 27)) * -7723592293110705685  # 0x94D049BB133111EB as int64
    z = z ^ (z >> 31)
    return int(z.sum().item())


def _bits(t):
    import torch

    return t.view(torch.int64) if t.dtype == torch.float64 else t


def _bad_model():
    import torch

    from paper_1704_08579_gb300 import learned

    p = learned.init_params(5)
    p[69760:] = 0.0
    p[86144 + 255] = 60.0  # only the last increment is large: every splitter at the sample minimum
    p[86144:86144 + 255] = -60.0
    return p.to(torch.float32)


@pytest.fixture(scope="module")
def trained():
    from paper_1704_08579_gb300 import learned

    qs_gpu()
    models = {}
    for kind in ("i32", "f64"):
        X, T = learned.training_set(kind, 1024, 1 << 16, seed=7)
        models[kind], _ = learned.train(X, T, steps=500, batch=128, lr=3e-4, seed=3)
    return models


def _make(name):
    import synth.device as sd

    if name == "zipf_i32_2p30":
        return sd.zipf_i32(1 << 30), "i32"
    if name == "gmix_i32_2p30":
        return sd.gauss_mix_i32(1 << 30), "i32"
    return sd.lognormal_f64(1 << 28), "f64"


@pytest.mark.parametrize("name", ["zipf_i32_2p30", "gmix_i32_2p30", "lognormal_f64_2p28"])
def test_full_learned_sort(name, trained):
    import torch

    qs = qs_gpu()
    x, kind = _make(name)
    h_in = _hash64(x)
    ref = x.clone()
    qs.sort(ref)
    torch.cuda.synchronize()
    assert bool((ref[1:] >= ref[:-1]).all()), "plain sort output not sorted"
    assert _hash64(ref) == h_in
    for model in (None, trained[kind], _bad_model()):
        d = x.clone()
        qs.sort_learned(d, model)
        torch.cuda.synchronize()
        st = qs.stats()
        assert st["bucket_max"] > 0
        assert torch.equal(_bits(d), _bits(ref)), "learned sort differs from the plain sort"
        del d
    host = x.cpu().numpy()
    got = ref.cpu().numpy()
    del x, ref
    torch.cuda.empty_cache()
    assert_keys_equal(got, oracle.sort_parallel(host))
