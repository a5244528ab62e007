"""Pins for the oracle's learned-splitter parts (CPU only).

MLP (1024 -> 64 -> 64 -> 256 softplus increments -> 255 cumulative quantiles):
  * central finite differences in double precision agree with the analytic
    gradient for a spread of parameters in every tensor (catches a dropped
    ReLU mask, a missing sigmoid, a wrong cumsum direction or normalisation);
  * closed form: with every weight zero and a constant output bias the 256
    increments are equal, so q_j = (j + 1) / 256 exactly;
  * outputs are non-decreasing inside [0, 1] (strictly, for moderate
    weights); a target equal to the model's own output gives zero loss and
    zero gradient.
Bucket partition: counts equal numpy's searchsorted (side='right') histogram
and the output equals a stable argsort of the bucket ids.
"""
import numpy as np
import pytest

import oracle
import synth

NP = oracle.mlp_nparams()
OFF_W1, OFF_B1 = 0, 64 * 1024
OFF_W2 = OFF_B1 + 64
OFF_B2 = OFF_W2 + 64 * 64
OFF_W3 = OFF_B2 + 64
OFF_B3 = OFF_W3 + 256 * 64


def _params(seed, scale=0.05):
    rng = np.random.default_rng(seed)
    p = rng.normal(0.0, scale, NP)
    p[OFF_B1:OFF_B1 + 64] = np.abs(p[OFF_B1:OFF_B1 + 64]) + 0.05  # keep most ReLUs active
    p[OFF_B2:OFF_B2 + 64] = np.abs(p[OFF_B2:OFF_B2 + 64]) + 0.05
    return p


def _batch(seed, b=3):
    rng = np.random.default_rng(seed)
    x = np.sort(rng.random((b, 1024)), axis=1)
    t = np.sort(rng.random((b, 255)), axis=1)
    return x, t


def test_parameter_count():
    assert NP == 64 * 1024 + 64 + 64 * 64 + 64 + 256 * 64 + 256


def test_closed_form_uniform_quantiles():
    p = np.zeros(NP)
    p[OFF_B3:OFF_B3 + 256] = 0.7
    x, _ = _batch(1, 2)
    q = oracle.mlp_forward(p, x)
    np.testing.assert_allclose(q, np.tile(np.arange(1, 256) / 256.0, (2, 1)), rtol=0, atol=1e-13)  # 256 additions of rounding


def test_outputs_monotone_in_unit_interval():
    # softplus increments are positive, though they can underflow to 0 in
    # floating point: the quantiles are non-decreasing and inside [0, 1].
    q = oracle.mlp_forward(_params(2, 0.3), _batch(3, 4)[0])
    assert np.all(q >= 0) and np.all(q <= 1) and np.all(np.diff(q, axis=1) >= 0)
    q = oracle.mlp_forward(_params(12, 0.02), _batch(13, 4)[0])
    assert np.all(q > 0) and np.all(q < 1) and np.all(np.diff(q, axis=1) > 0)


def test_zero_error_zero_gradient():
    p = _params(4)
    x, _ = _batch(5, 2)
    t = oracle.mlp_forward(p, x)
    loss, g = oracle.mlp_loss_grad(p, x, t)
    assert loss < 1e-30 and np.max(np.abs(g)) < 1e-15


@pytest.mark.parametrize("lo,hi", [(OFF_W1, OFF_B1), (OFF_B1, OFF_W2), (OFF_W2, OFF_B2), (OFF_B2, OFF_W3),
                                   (OFF_W3, OFF_B3), (OFF_B3, NP)])
def test_gradient_finite_differences(lo, hi):
    p = _params(6)
    x, t = _batch(7)
    _, g = oracle.mlp_loss_grad(p, x, t)
    rng = np.random.default_rng(lo)
    idx = rng.choice(np.arange(lo, hi), size=min(12, hi - lo), replace=False)
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (oracle.mlp_loss_grad(pp, x, t)[0] - oracle.mlp_loss_grad(pm, x, t)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-7 + 1e-5 * abs(fd), (i, fd, g[i])


@pytest.mark.parametrize("dtype", [np.int32, np.float64])
def test_bucket_partition(dtype):
    if dtype == np.int32:
        x = synth.mod_i32(50_001, 8, 1000)
        spl = np.sort(synth.mod_i32(255, 9, 1000))
    else:
        x = synth.uniform_f64(50_001, 10)
        spl = np.sort(synth.uniform_f64(255, 11))
    out, counts = oracle.bucket(x, spl)
    b = np.searchsorted(spl, x, side="right")
    np.testing.assert_array_equal(counts, np.bincount(b, minlength=256))
    np.testing.assert_array_equal(out, x[np.argsort(b, kind="stable")])


def test_adam_first_step_closed_form():
    """At step 1 with zero moments the bias-corrected update is lr * g / (|g| + eps)."""
    rng = np.random.default_rng(14)
    p = rng.normal(size=1000)
    g = rng.normal(size=1000)
    z = np.zeros(1000)
    p1, m1, v1 = oracle.adam_step(p, g, z, z, 1, 0.01)
    np.testing.assert_allclose(p1, p - 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(m1, 0.1 * g, rtol=1e-14)
    np.testing.assert_allclose(v1, 0.001 * g * g, rtol=1e-12)
    # a second step with the same gradient keeps moving the same way
    p2, _, _ = oracle.adam_step(p1, g, m1, v1, 2, 0.01)
    assert np.all(np.sign(p1 - p2) == np.sign(g))


def test_adam_constant_gradient_closed_form():
    """With the same gradient at every step, the bias-corrected moments equal
    g and g^2 exactly, so every step moves each parameter by lr * g / (|g| +
    eps) -- a wrong bias-correction power or a swapped beta shows up by step 2."""
    rng = np.random.default_rng(15)
    p0 = rng.normal(size=500)
    g = rng.normal(size=500)
    p, m, v = p0.copy(), np.zeros(500), np.zeros(500)
    step = 0.003 * g / (np.abs(g) + 1e-8)
    for t in range(1, 9):
        p, m, v = oracle.adam_step(p, g, m, v, t, 0.003)
        np.testing.assert_allclose(p, p0 - t * step, rtol=1e-9, atol=1e-12)
        np.testing.assert_allclose(m, (1 - 0.9 ** t) * g, rtol=1e-12)
        np.testing.assert_allclose(v, (1 - 0.999 ** t) * g * g, rtol=1e-9)
