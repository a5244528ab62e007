"""The device-side generators of the skewed workloads reproduce the host
generators' SplitMix64 streams bit for bit (run here on torch's CPU device)."""
import numpy as np
import pytest

import synth


def test_device_splitmix_matches_host():
    pytest.importorskip("torch")
    import synth.device as sd

    for seed, start in ((0, 0), (0x5EED0008, 1000), ((1 << 64) - 1, (1 << 33) + 5)):
        a = synth.splitmix64(seed, start, 4099).view(np.int64)
        b = sd.splitmix64(seed, start, 4099, device="cpu").numpy()
        np.testing.assert_array_equal(a, b)


def test_device_generators_match_host():
    pytest.importorskip("torch")
    import synth.device as sd

    n = (1 << 16) + 3
    np.testing.assert_array_equal(sd.zipf_i32(n, device="cpu").numpy(), synth.zipf_i32(n))
    g = sd.gauss_mix_i32(n, device="cpu").numpy()
    assert np.count_nonzero(g != synth.gauss_mix_i32(n)) <= n // 1000
    np.testing.assert_allclose(sd.lognormal_f64(n, device="cpu").numpy(), synth.lognormal_f64(n), rtol=1e-13)
