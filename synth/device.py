"""The skewed learned-splitter workloads generated on the GPU (torch), for
array sizes where the host generators would take minutes (2^28 .. 2^30 keys).

Same recipes and the same SplitMix64 streams as ``synth.zipf_i32``,
``synth.gauss_mix_i32`` and ``synth.lognormal_f64``: the counter-based draws
are computed in 64-bit integer arithmetic (wrapping multiplies, logical
shifts by masking) and agree bit for bit with the host's; the Zipf keys are
therefore identical, while the Box-Muller normals (log1p, sqrt, cos on the
device) may differ from the host's in the last bit.  Like the host module,
this one holds none of the sorting method's arithmetic.
"""
from __future__ import annotations

import math

from . import SEEDS, gauss_mix_params, zipf_cdf

_CHUNK = 1 << 24


def _i64(u: int) -> int:
    """A uint64 constant as the int64 with the same bits."""
    u &= 0xFFFFFFFFFFFFFFFF
    return u - (1 << 64) if u >= 1 << 63 else u


_GOLDEN = _i64(0x9E3779B97F4A7C15)
_M1 = _i64(0xBF58476D1CE4E5B9)
_M2 = _i64(0x94D049BB133111EB)


def _srl(z, k: int):
    """Logical right shift of int64 bit patterns."""
    return (z >> k) & ((1 << (64 - k)) - 1)


def splitmix64(seed: int, start: int, count: int, device="cuda"):
    """Outputs start .. start+count-1 of the stream, as int64 tensors holding the uint64 bits."""
    import torch

    idx = torch.arange(start + 1, start + count + 1, dtype=torch.int64, device=device)
    z = idx * _GOLDEN + _i64(seed)
    z = (z ^ _srl(z, 30)) * _M1
    z = (z ^ _srl(z, 27)) * _M2
    return z ^ _srl(z, 31)


def _u53(z):
    import torch

    return _srl(z, 11).to(torch.float64) * (1.0 / 9007199254740992.0)


def _normal(seed: int, a: int, b: int, device):
    import torch

    u1 = _u53(splitmix64(seed, a, b - a, device))
    u2 = _u53(splitmix64(seed ^ 0xB0B, a, b - a, device))
    return torch.sqrt(-2.0 * torch.log1p(-u1)) * torch.cos(2.0 * math.pi * u2)


def zipf_i32(n: int, seed: int | None = None, s: float = 1.2, nvals: int = 1 << 24, device="cuda"):
    import torch

    seed = SEEDS["c5_zipf_i32"] if seed is None else seed
    cdf = torch.from_numpy(zipf_cdf(s, nvals)).to(device)
    mult = (2654435761 | 1) % nvals
    out = torch.empty(n, dtype=torch.int32, device=device)
    for a in range(0, n, _CHUNK):
        b = min(n, a + _CHUNK)
        rank = torch.searchsorted(cdf, _u53(splitmix64(seed, a, b - a, device)), right=True).clamp_(max=nvals - 1)
        code = (rank * mult + 12345) % nvals
        out[a:b] = (code * 256 - (1 << 31)).to(torch.int32)
    return out


def gauss_mix_i32(n: int, seed: int | None = None, k: int = 8, device="cuda"):
    import torch

    seed = SEEDS["c5_gmix_i32"] if seed is None else seed
    means, sig, cw = gauss_mix_params(seed, k)
    means, sig, cw = (torch.from_numpy(v).to(device) for v in (means, sig, cw))
    out = torch.empty(n, dtype=torch.int32, device=device)
    for a in range(0, n, _CHUNK):
        b = min(n, a + _CHUNK)
        u = _u53(splitmix64(seed ^ 0xA11, a, b - a, device))
        comp = torch.searchsorted(cw, u, right=True).clamp_(max=k - 1)
        x = torch.round(means[comp] + sig[comp] * _normal(seed, a, b, device))
        out[a:b] = x.clamp_(-2147483648.0, 2147483647.0).to(torch.int32)
    return out


def lognormal_f64(n: int, seed: int | None = None, sigma: float = 2.0, device="cuda"):
    import torch

    seed = SEEDS["c5_lognormal_f64"] if seed is None else seed
    out = torch.empty(n, dtype=torch.float64, device=device)
    for a in range(0, n, _CHUNK):
        b = min(n, a + _CHUNK)
        out[a:b] = torch.exp(sigma * _normal(seed, a, b, device))
    return out
