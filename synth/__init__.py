"""Seeded synthetic inputs shared by the oracle side and the CUDA side.

This module only produces numbers; it holds none of the sorting method's
arithmetic (no comparisons against pivots, no partitioning, no sorting).
Every generator is counter based: element ``i`` of a stream with seed ``s``
is ``splitmix64(s, i)``, so any slice of any array can be regenerated
independently and both sides receive the same bytes.

SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
generators", OOPSLA 2014): the state advances by the golden-ratio increment
0x9E3779B97F4A7C15 and each output is the state passed through the
variant-13 mixing function (shifts 30, 27, 31 and two odd multipliers).

Workload shapes follow the paper's experiments (random values, sizes
2^1 .. 2^30, Section IV) and the five benchmark configurations: uniform /
sorted / reverse / few-unique FP64, int32 key-value pairs with value =
original index, batched uneven segments, and the skewed distributions used
by the learned-splitter path.
"""
from __future__ import annotations

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_CHUNK = 1 << 22

# One seed per (configuration, distribution); fixed so every run sees the same bytes.
SEEDS = {
    "c1_uniform_i32": 0x5EED0001,
    "c2_uniform_f64": 0x5EED0002,
    "c2_few_f64": 0x5EED0003,
    "c3_uniform_kv": 0x5EED0004,
    "c3_mod1000_kv": 0x5EED0005,
    "c3_sorted_kv": 0x5EED0006,
    "c4_segments": 0x5EED0007,
    "c5_zipf_i32": 0x5EED0008,
    "c5_gmix_i32": 0x5EED0009,
    "c5_lognormal_f64": 0x5EED000A,
}


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Outputs ``start .. start+count-1`` of the SplitMix64 stream seeded with ``seed``."""
    idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + idx * _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def _chunks(n: int):
    for s in range(0, n, _CHUNK):
        yield s, min(n, s + _CHUNK)


def _u53(z: np.ndarray) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits."""
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def uniform_i32(n: int, seed: int) -> np.ndarray:
    """Keys uniform over the full signed 32-bit range (top 32 bits of each draw)."""
    out = np.empty(n, dtype=np.int32)
    for a, b in _chunks(n):
        out[a:b] = (splitmix64(seed, a, b - a) >> np.uint64(32)).astype(np.uint32).view(np.int32)
    return out


def mod_i32(n: int, seed: int, m: int) -> np.ndarray:
    """Keys ``(uint32)draw % m``: values 0 .. m-1, heavy duplicates for small m."""
    out = np.empty(n, dtype=np.int32)
    for a, b in _chunks(n):
        u = (splitmix64(seed, a, b - a) >> np.uint64(32)).astype(np.uint32)
        out[a:b] = (u % np.uint32(m)).astype(np.int32)
    return out


def ascending_i32(n: int, seed: int) -> np.ndarray:
    """Non-decreasing int32 keys spread over the full range: key_i = -2^31 + floor((i + u_i) 2^32 / n)."""
    out = np.empty(n, dtype=np.int32)
    for a, b in _chunks(n):
        i = np.arange(a, b, dtype=np.uint64)
        frac = splitmix64(seed, a, b - a) >> np.uint64(32)
        v = (i * np.uint64(1 << 32) + frac) // np.uint64(max(n, 1))
        out[a:b] = (v.astype(np.int64) - (1 << 31)).astype(np.int32)
    return out


def uniform_f64(n: int, seed: int, lo: float = -1e6, hi: float = 1e6) -> np.ndarray:
    """Doubles uniform in [lo, hi); -0.0 is mapped to +0.0 (no NaN can occur)."""
    out = np.empty(n, dtype=np.float64)
    for a, b in _chunks(n):
        out[a:b] = lo + (hi - lo) * _u53(splitmix64(seed, a, b - a))
    out += 0.0  # -0.0 + 0.0 == +0.0 under round-to-nearest
    return out


def ascending_f64(n: int, seed: int, lo: float = -1e6, hi: float = 1e6) -> np.ndarray:
    """Non-decreasing doubles in [lo, hi): x_i = lo + (hi - lo) (i + u_i) / n (monotone rounding)."""
    out = np.empty(n, dtype=np.float64)
    for a, b in _chunks(n):
        i = np.arange(a, b, dtype=np.float64)
        out[a:b] = lo + (hi - lo) * ((i + _u53(splitmix64(seed, a, b - a))) / max(n, 1))
    out += 0.0
    return out


def few_unique_f64(n: int, seed: int, k: int = 16, lo: float = -1e6, hi: float = 1e6) -> np.ndarray:
    """k distinct doubles drawn once, then each element picks one uniformly."""
    table = uniform_f64(k, seed ^ 0xF00D, lo, hi)
    out = np.empty(n, dtype=np.float64)
    for a, b in _chunks(n):
        idx = (splitmix64(seed, a, b - a) >> np.uint64(32)) % np.uint64(k)
        out[a:b] = table[idx.astype(np.int64)]
    return out


def f64_config(dist: str, n: int, seed: int | None = None) -> np.ndarray:
    """The four FP64 distributions of the full-sort workload: uniform, sorted, reverse, few."""
    if dist == "uniform":
        return uniform_f64(n, SEEDS["c2_uniform_f64"] if seed is None else seed)
    if dist == "sorted":
        return ascending_f64(n, SEEDS["c2_uniform_f64"] if seed is None else seed)
    if dist == "reverse":
        return ascending_f64(n, SEEDS["c2_uniform_f64"] if seed is None else seed)[::-1].copy()
    if dist == "few":
        return few_unique_f64(n, SEEDS["c2_few_f64"] if seed is None else seed)
    raise ValueError(dist)


def kv_config(dist: str, n: int, seed: int | None = None):
    """int32 keys + int32 values (value = original index) for the key/value workload."""
    if dist == "uniform":
        keys = uniform_i32(n, SEEDS["c3_uniform_kv"] if seed is None else seed)
    elif dist == "mod1000":
        keys = mod_i32(n, SEEDS["c3_mod1000_kv"] if seed is None else seed, 1000)
    elif dist == "sorted":
        keys = ascending_i32(n, SEEDS["c3_sorted_kv"] if seed is None else seed)
    elif dist == "reverse":
        keys = ascending_i32(n, SEEDS["c3_sorted_kv"] if seed is None else seed)[::-1].copy()
    else:
        raise ValueError(dist)
    vals = np.arange(n, dtype=np.int32)
    return keys, vals


def segment_sizes(nseg: int, seed: int, lo: int = 16, hi: int = 1 << 18) -> np.ndarray:
    """Segment lengths floor(exp(U[ln lo, ln hi])) (log-uniform), as int64."""
    u = _u53(splitmix64(seed, 0, nseg))
    return np.floor(np.exp(np.log(lo) + (np.log(hi) - np.log(lo)) * u)).astype(np.int64)


def segments_i32(nseg: int, seed: int | None = None, lo: int = 16, hi: int = 1 << 18):
    """Concatenated uniform int32 arrays of log-uniform sizes plus int64 offsets (nseg + 1)."""
    seed = SEEDS["c4_segments"] if seed is None else seed
    sizes = segment_sizes(nseg, seed ^ 0x5E65, lo, hi)
    offsets = np.zeros(nseg + 1, dtype=np.int64)
    np.cumsum(sizes, out=offsets[1:])
    keys = uniform_i32(int(offsets[-1]), seed)
    return keys, offsets


def _normal(seed: int, a: int, b: int) -> np.ndarray:
    """Standard normals by Box-Muller from two independent uniform streams."""
    u1 = _u53(splitmix64(seed, a, b - a))
    u2 = _u53(splitmix64(seed ^ 0xB0B, a, b - a))
    r = np.sqrt(-2.0 * np.log1p(-u1))  # 1 - u1 in (0, 1]
    return r * np.cos(2.0 * np.pi * u2)


def zipf_i32(n: int, seed: int | None = None, s: float = 1.2, nvals: int = 1 << 24) -> np.ndarray:
    """Zipf(s) ranks over 1..nvals by inverse CDF, mapped by a seeded bijection onto {k*256 - 2^31}."""
    seed = SEEDS["c5_zipf_i32"] if seed is None else seed
    cdf = zipf_cdf(s, nvals)
    mult = np.int64(2654435761 | 1) % np.int64(nvals)  # odd => bijection mod 2^24
    out = np.empty(n, dtype=np.int32)
    for a, b in _chunks(n):
        rank = np.searchsorted(cdf, _u53(splitmix64(seed, a, b - a)), side="right")
        rank = np.minimum(rank, nvals - 1).astype(np.int64)
        code = (rank * mult + 12345) % nvals
        out[a:b] = (code * 256 - (1 << 31)).astype(np.int32)
    return out


def gauss_mix_params(seed: int, k: int = 8):
    """Component means U[-1.5e9, 1.5e9], sigmas log-U[1e5, 1e8] and cumulative weights of the mixture."""
    p = _u53(splitmix64(seed ^ 0xC0FFEE, 0, 3 * k))
    means = -1.5e9 + 3e9 * p[:k]
    sig = np.exp(np.log(1e5) + (np.log(1e8) - np.log(1e5)) * p[k:2 * k])
    wts = 0.5 + p[2 * k:]
    return means, sig, np.cumsum(wts / wts.sum())


def gauss_mix_i32(n: int, seed: int | None = None, k: int = 8) -> np.ndarray:
    """Mixture of k Gaussians (means U[-1.5e9, 1.5e9], sigma log-U[1e5, 1e8]), rounded, clipped to int32."""
    seed = SEEDS["c5_gmix_i32"] if seed is None else seed
    means, sig, cw = gauss_mix_params(seed, k)
    out = np.empty(n, dtype=np.int32)
    for a, b in _chunks(n):
        comp = np.minimum(np.searchsorted(cw, _u53(splitmix64(seed ^ 0xA11, a, b - a)), side="right"), k - 1)
        x = np.rint(means[comp] + sig[comp] * _normal(seed, a, b))
        out[a:b] = np.clip(x, -2147483648.0, 2147483647.0).astype(np.int32)
    return out


def zipf_cdf(s: float = 1.2, nvals: int = 1 << 24) -> np.ndarray:
    w = np.arange(1, nvals + 1, dtype=np.float64) ** (-s)
    cdf = np.cumsum(w)
    cdf /= cdf[-1]
    return cdf


def lognormal_f64(n: int, seed: int | None = None, sigma: float = 2.0) -> np.ndarray:
    """exp(sigma * N(0, 1)) doubles (mu = 0)."""
    seed = SEEDS["c5_lognormal_f64"] if seed is None else seed
    out = np.empty(n, dtype=np.float64)
    for a, b in _chunks(n):
        out[a:b] = np.exp(sigma * _normal(seed, a, b))
    return out
