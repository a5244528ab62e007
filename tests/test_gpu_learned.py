"""Learned-splitter form on the GPU against the oracle.

* The splitter MLP: forward outputs, the loss and every parameter tensor's
  gradient against the double-precision oracle (FP32 kernels: relative L2
  error per tensor below 1e-3), and the Adam step against the oracle's.
* The sketch: sorted, drawn from the input, min-max scaled.
* The 256-way bucket pass with the caller's splitters: bucket offsets exactly
  the oracle's, each bucket the oracle's multiset, every key inside its
  splitter interval.
* The learned sort (trained, untrained, random and sampled splitters) gives
  the oracle's sorted keys bit for bit, including degenerate splitter sets
  that put everything in one bucket (the plain-method fallback).
* Training on sort-generated quantiles with the library's own kernels lowers
  the quantile-position error on held-out arrays, and the learned splitters
  give a lower bucket-imbalance error (what the plain method measures) than
  the same sketch's sampled splitters.
"""
import numpy as np
import pytest

import oracle
import synth
from qs_testutil import assert_keys_equal, qs_gpu, to_dev

pytestmark = pytest.mark.gpu

NP = 86400
W1, B1, W2, B2, W3, B3 = 0, 65536, 65600, 69696, 69760, 86144
SLICES = {"W1": (W1, B1), "b1": (B1, W2), "W2": (W2, B2), "b2": (B2, W3), "W3": (W3, B3), "b3": (B3, NP)}


def _params(seed: int, w3: float = 0.3) -> np.ndarray:
    """Random parameters (float32) with a non-zero last layer, so every term of the network matters."""
    p = np.empty(NP, dtype=np.float64)
    a1, a2, a3 = np.sqrt(6.0 / 1024), np.sqrt(6.0 / 64), w3
    p[W1:B1] = synth.uniform_f64(B1 - W1, seed, -a1, a1)
    p[B1:W2] = synth.uniform_f64(W2 - B1, seed + 1, -0.1, 0.1)
    p[W2:B2] = synth.uniform_f64(B2 - W2, seed + 2, -a2, a2)
    p[B2:W3] = synth.uniform_f64(W3 - B2, seed + 3, -0.1, 0.1)
    p[W3:B3] = synth.uniform_f64(B3 - W3, seed + 4, -a3, a3)
    p[B3:NP] = synth.uniform_f64(NP - B3, seed + 5, -1.0, 1.0)
    return p.astype(np.float32)


def _sketches(batch: int, seed: int) -> np.ndarray:
    """Sorted [0, 1] sketches of varied shapes (powers of an ascending ramp)."""
    x = np.empty((batch, 1024), dtype=np.float32)
    for b in range(batch):
        r = synth.ascending_f64(1024, seed + b, 0.0, 1.0)
        r = (r - r[0]) / (r[-1] - r[0])
        x[b] = r ** (0.3 + 0.4 * b)
    return x


def _targets(batch: int, seed: int) -> np.ndarray:
    base = (np.arange(255) + 1) / 256.0
    t = np.empty((batch, 255), dtype=np.float32)
    for b in range(batch):
        t[b] = np.clip(base + synth.uniform_f64(255, seed + b, -0.01, 0.01), 0, 1)
    return t


def _rel_l2(got, exp):
    return float(np.linalg.norm(got - exp) / max(np.linalg.norm(exp), 1e-30))


# ---------------------------------------------------------------------------
# MLP kernels vs the oracle
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("batch", [1, 9])
def test_mlp_forward_matches_oracle(batch):
    qs = qs_gpu()
    p = _params(11)
    x = _sketches(batch, 100)
    q = qs.mlp_forward(to_dev(p), to_dev(x)).cpu().numpy()
    qo = oracle.mlp_forward(p.astype(np.float64), x.astype(np.float64))
    assert q.shape == (batch, 255)
    np.testing.assert_allclose(q, qo, rtol=0, atol=5e-5)
    assert np.all(np.diff(q, axis=1) >= 0), "quantile positions must be non-decreasing"


def test_mlp_forward_untrained_is_even():
    """Last layer zero: q_j = (j + 1) / 256 whatever the sketch (the sampled splitters)."""
    qs = qs_gpu()
    p = _params(12)
    p[W3:NP] = 0
    q = qs.mlp_forward(to_dev(p), to_dev(_sketches(3, 200))).cpu().numpy()
    np.testing.assert_allclose(q, np.tile((np.arange(255) + 1) / 256.0, (3, 1)), rtol=0, atol=1e-6)


@pytest.mark.parametrize("batch", [1, 9, 64])
def test_mlp_gradient_matches_oracle(batch):
    import torch

    qs = qs_gpu()
    p = _params(21)
    x = _sketches(batch, 300)
    t = _targets(batch, 400)
    dp, dx, dt = to_dev(p), to_dev(x), to_dev(t)
    act = torch.empty(batch, 640, dtype=torch.float32, device="cuda")
    work = torch.empty(batch, 384, dtype=torch.float32, device="cuda")
    grad = torch.empty(NP, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    qs.mlp_forward(dp, dx, act)
    qs.mlp_backward(dp, dx, dt, act, work, grad, loss)
    g = grad.cpu().numpy().astype(np.float64)
    lo, go = oracle.mlp_loss_grad(p.astype(np.float64), x.astype(np.float64), t.astype(np.float64))
    assert abs(float(loss.item()) - lo) <= 1e-4 * lo
    for name, (a, b) in SLICES.items():
        err = _rel_l2(g[a:b], go[a:b])
        assert err < 1e-3, "%s: relative L2 error %.3g" % (name, err)


def test_adam_matches_oracle():
    import torch

    qs = qs_gpu()
    p = _params(31)
    gs = [synth.uniform_f64(NP, 500 + k, -1e-2, 1e-2).astype(np.float32) for k in range(3)]
    dp = to_dev(p)
    m = torch.zeros(NP, dtype=torch.float32, device="cuda")
    v = torch.zeros(NP, dtype=torch.float32, device="cuda")
    po, mo, vo = p.astype(np.float64), np.zeros(NP), np.zeros(NP)
    for k, g in enumerate(gs, start=1):
        qs.mlp_adam(dp, to_dev(g), m, v, k, 1e-3)
        po, mo, vo = oracle.adam_step(po, g.astype(np.float64), mo, vo, k, 1e-3)
        np.testing.assert_allclose(dp.cpu().numpy(), po, rtol=1e-6, atol=1e-7)
        np.testing.assert_allclose(m.cpu().numpy(), mo, rtol=1e-5, atol=5e-10)  # m cancels to ~0 in places
        np.testing.assert_allclose(v.cpu().numpy(), vo, rtol=1e-5, atol=1e-14)


# ---------------------------------------------------------------------------
# Sketch and bucket pass
# ---------------------------------------------------------------------------
def _keys(kind: str, n: int, seed_shift: int = 0):
    if kind == "zipf":
        return synth.zipf_i32(n, synth.SEEDS["c5_zipf_i32"] + seed_shift)
    if kind == "gmix":
        return synth.gauss_mix_i32(n, synth.SEEDS["c5_gmix_i32"] + seed_shift)
    if kind == "lognormal":
        return synth.lognormal_f64(n, synth.SEEDS["c5_lognormal_f64"] + seed_shift)
    if kind == "uniform_i32":
        return synth.uniform_i32(n, 0x1234 + seed_shift)
    return synth.uniform_f64(n, 0x4321 + seed_shift)


@pytest.mark.parametrize("kind", ["zipf", "gmix", "lognormal", "uniform_f64"])
@pytest.mark.parametrize("n", [1024, 5000, (1 << 20) + 77])
def test_sketch_properties(kind, n):
    qs = qs_gpu()
    x = _keys(kind, n)
    d = to_dev(x)
    sk, mm, smp = qs.sketch(d)
    sk, mm, smp = sk.cpu().numpy(), mm.cpu().numpy(), smp.cpu().numpy()
    assert_keys_equal(d.cpu().numpy(), x)  # input untouched
    assert np.all(np.diff(smp) >= 0)
    assert np.all(np.isin(smp, x)), "sample keys must come from the input"
    assert mm[0] == float(smp[0]) and mm[1] == float(smp[-1])
    assert np.all(np.diff(sk) >= 0) and sk[0] == 0.0
    if mm[1] > mm[0]:
        assert sk[-1] == 1.0
        np.testing.assert_allclose(sk, (smp.astype(np.float64) - mm[0]) / (mm[1] - mm[0]), rtol=0, atol=1e-6)


def _check_bucket(x, spl, got, off):
    out, counts = oracle.bucket(x, spl)
    exp_off = np.concatenate(([0], np.cumsum(counts)))
    np.testing.assert_array_equal(off, exp_off)
    for b in range(spl.size + 1):
        a, e = exp_off[b], exp_off[b + 1]
        if a == e:
            continue
        assert_keys_equal(np.sort(got[a:e], kind="stable"), np.sort(out[a:e], kind="stable"))
        if b > 0:
            assert np.all(got[a:e] >= spl[b - 1])
        if b < spl.size:
            assert np.all(got[a:e] < spl[b])


@pytest.mark.parametrize("kind", ["zipf", "gmix", "lognormal", "uniform_i32"])
@pytest.mark.parametrize("nsplit", [1, 7, 255])
def test_bucket_pass_matches_oracle(kind, nsplit):
    qs = qs_gpu()
    n = (1 << 20) + 12345
    x = _keys(kind, n, 1)
    # splitters: sorted draws from the input, with repeats for the skewed kinds
    idx = (synth.splitmix64(0xB0C, 0, nsplit) % np.uint64(n)).astype(np.int64)
    spl = np.sort(x[idx])
    d = to_dev(x)
    off = qs.bucket(d, to_dev(spl)).cpu().numpy()
    _check_bucket(x, spl, d.cpu().numpy(), off)


@pytest.mark.parametrize("n", [0, 1, 255, 4097])
def test_bucket_pass_small_and_edges(n):
    qs = qs_gpu()
    x = synth.mod_i32(n, 0x77, 50)
    spl = np.array([-5, 0, 0, 10, 25, 25, 49, 60], dtype=np.int32)
    d = to_dev(x)
    off = qs.bucket(d, to_dev(spl)).cpu().numpy()
    _check_bucket(x, spl, d.cpu().numpy(), off)


def test_bucket_pass_extreme_splitters_f64():
    """Splitters at the extremes of the key type: everything lands in the middle bucket."""
    qs = qs_gpu()
    x = synth.uniform_f64(300000, 0x99)
    spl = np.array([-np.inf, -1e300, 1e300, np.inf], dtype=np.float64)
    d = to_dev(x)
    off = qs.bucket(d, to_dev(spl)).cpu().numpy()
    _check_bucket(x, spl, d.cpu().numpy(), off)


# ---------------------------------------------------------------------------
# Learned sort: exact output whatever the splitters
# ---------------------------------------------------------------------------
def _model(which: str, seed: int = 41):
    import torch

    if which == "sampled":
        return None
    p = _params(seed, w3=0.3 if which == "random" else 0.0)
    if which == "untrained":
        p[W3:NP] = 0
    if which == "collapse":
        # only the last increment is large: every q_j ~ 0, every splitter is
        # the smallest sample key, so the last bucket holds almost all keys
        p[W3:NP] = 0
        p[B3 + 255] = 60.0
        p[B3:B3 + 255] = -60.0
    if which == "front":
        # only the first increment is large: every q_j ~ 1, every splitter is
        # the largest sample key, so the first bucket holds almost all keys
        p[W3:NP] = 0
        p[B3] = 60.0
        p[B3 + 1:NP] = -60.0
    return torch.from_numpy(p).to("cuda")


@pytest.fixture(params=[1, 2], ids=["one_level", "two_levels"])
def levels(request):
    """QS_OPT_BUCKET_LEVELS for the test (one 256-way bucket pass, or a
    second one inside every bucket); restored to the default afterwards."""
    qs = qs_gpu()
    qs.set_option("bucket_levels", request.param)
    yield request.param
    qs.set_option("bucket_levels", 0)


@pytest.mark.parametrize("kind", ["zipf", "gmix", "lognormal"])
@pytest.mark.parametrize("which", ["sampled", "untrained", "random", "collapse", "front"])
def test_learned_sort_matches_oracle(kind, which, levels):
    qs = qs_gpu()
    n = (1 << 20) + 4321
    x = _keys(kind, n, 2)
    d = to_dev(x)
    qs.sort_learned(d, _model(which))
    st = qs.stats()
    assert_keys_equal(d.cpu().numpy(), oracle.sort(x))
    assert st["bucket_max"] >= (n + 255) // 256
    if which in ("collapse", "front"):
        assert st["bucket_over"] >= 1, "a degenerate model must trip the size bound"


@pytest.mark.parametrize("n", [0, 1, 1000, (1 << 16) - 1, 1 << 16, (1 << 16) + 1, 3 << 18, (1 << 22) + 65537])
def test_learned_sort_sizes(n, levels):
    qs = qs_gpu()
    x = synth.uniform_i32(n, 0x515)
    d = to_dev(x)
    qs.sort_learned(d, _model("random"))
    assert_keys_equal(d.cpu().numpy(), oracle.sort(x))


@pytest.mark.parametrize("dtype", ["i32", "f64"])
def test_learned_sort_degenerate_inputs(dtype, levels):
    """All keys equal, sorted and reverse-sorted input, two distinct keys."""
    qs = qs_gpu()
    n = 300000
    if dtype == "i32":
        cases = [np.full(n, 7, np.int32), synth.ascending_i32(n, 1), synth.ascending_i32(n, 2)[::-1].copy(),
                 synth.mod_i32(n, 3, 2)]
    else:
        cases = [np.full(n, -2.5), synth.ascending_f64(n, 1), synth.ascending_f64(n, 2)[::-1].copy(),
                 synth.few_unique_f64(n, 3, 2)]
    for x in cases:
        for which in ("sampled", "random"):
            d = to_dev(x)
            qs.sort_learned(d, _model(which))
            assert_keys_equal(d.cpu().numpy(), oracle.sort(x))


def test_learned_sort_rejects_bad_params():
    import torch

    qs = qs_gpu()
    d = to_dev(synth.uniform_i32(1 << 17, 5))
    with pytest.raises(ValueError):
        qs.sort_learned(d, torch.zeros(10, dtype=torch.float32, device="cuda"))
    with pytest.raises(TypeError):
        qs.sort_learned(d.to(torch.int64), None)


# ---------------------------------------------------------------------------
# Training with the library's kernels, and what it gains
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("kind", ["i32", "f64"])
def test_training_gain(kind):
    """Trained with the library's kernels on sort-generated (sketch, exact
    quantile) pairs, the network predicts the quantile positions of held-out
    arrays markedly better than the untrained one (even positions), and the
    learned splitters cut fresh arrays into more even buckets than the same
    sketch's sampled splitters: the bucket-imbalance error (bucket_dev / 2nB,
    the total variation distance from an even split) that the plain method
    measures."""
    from paper_1704_08579_gb300 import learned

    qs_gpu()
    X, T = learned.training_set(kind, 4096, 1 << 16, seed=7)
    p, losses = learned.train(X, T, steps=3000, batch=128, lr=3e-4, seed=3)
    assert losses[-1] < losses[0]
    Xh, Th = learned.training_set(kind, 128, 1 << 16, seed=99)
    e_trained = learned.position_error(p, Xh, Th)
    e_init = learned.position_error(learned.init_params(0), Xh, Th)
    cmp = learned.compare(p, kind, 16, 1 << 20, seed=12345)
    print("\n%s position error: trained %.3g untrained %.3g" % (kind, e_trained, e_init))
    for fam, d in cmp.items():
        print("%s %-9s imbalance error: learned %.4f untrained %.4f sampled %.4f"
              % (kind, fam, d["learned"], d["untrained"], d["sampled"]))
    # measured: trained / untrained = 0.60 (int32 families), 0.93 (FP64 families)
    assert e_trained < {"i32": 0.8, "f64": 0.97}[kind] * e_init
    ml = float(np.mean([d["learned"] for d in cmp.values()]))
    ms = float(np.mean([d["sampled"] for d in cmp.values()]))
    assert ml < ms


@pytest.mark.parametrize("dtype", ["i32", "f64"])
def test_two_level_buckets_skewed_and_chunked(dtype):
    """Second bucket level: buckets of very different sizes (Zipf / lognormal
    keys, so some buckets span many chunks of the second-level passes and
    others are empty), a heavy key that fills whole sub-buckets, and sizes
    that leave a ragged last chunk -- against the oracle."""
    qs = qs_gpu()
    try:
        qs.set_option("bucket_levels", 2)
        for n in ((1 << 21) + 12345, (1 << 23) + 3):
            if dtype == "i32":
                x = synth.zipf_i32(n, 17)
            else:
                x = synth.lognormal_f64(n, 18)
            for which in ("sampled", "random"):
                d = to_dev(x)
                qs.sort_learned(d, _model(which))
                assert_keys_equal(d.cpu().numpy(), oracle.sort(x))
        heavy = np.where(synth.mod_i32(1 << 20, 19, 3) == 0, 5, synth.uniform_i32(1 << 20, 20)).astype(np.int32)
        if dtype == "f64":
            heavy = heavy.astype(np.float64) * 0.5
        d = to_dev(heavy)
        qs.sort_learned(d, _model("sampled"))
        assert_keys_equal(d.cpu().numpy(), oracle.sort(heavy))
    finally:
        qs.set_option("bucket_levels", 0)
