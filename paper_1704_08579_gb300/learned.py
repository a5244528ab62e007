"""Training and evaluation of the splitter MLP (learned form of the sort).

The network is trained on (sketch, exact quantile) pairs that the sort itself
generates: for each training array the library computes the 1024-key sketch
(qs_sketch_*) and sorts the array (qs_sort_*); the targets are the keys at
ranks floor((j+1) n / 256), j = 0..254, of the sorted array, expressed as
positions along the sorted sample (the space the model predicts in: a key that
occurs in the sample maps to the middle of its run there, a key between two
sample keys to the linear interpolation between their positions).  The
forward, backward and Adam steps are the library's own kernels
(qs_mlp_forward / qs_mlp_backward / qs_mlp_adam); torch only holds buffers and
draws the training arrays.

The untrained network (last layer zero) outputs q_j = (j+1)/256, i.e. the
sampled splitters; training moves it from there.
"""
from __future__ import annotations

import math

import paper_1704_08579_gb300 as qs

NQ = 255


def _torch():
    import torch

    return torch


# ---------------------------------------------------------------------------
# Training arrays: distribution families with random shape parameters.
# ---------------------------------------------------------------------------
def draw_array(kind: str, family: str, n: int, gen):
    """One training array of n keys (CUDA tensor), family in zipf / gmix /
    uniform / normal (int32) or lognormal / gmix / normal / uniform (f64)."""
    torch = _torch()
    dev = "cuda"
    u = lambda *s: torch.rand(*s, generator=gen, device=dev, dtype=torch.float64)  # noqa: E731
    if kind == "i32":
        if family == "zipf":
            s = 1.05 + 0.55 * float(u(1))
            nv = 1 << int(16 + 8 * float(u(1)))
            w = torch.arange(1, nv + 1, device=dev, dtype=torch.float64) ** (-s)
            cdf = torch.cumsum(w, 0)
            cdf /= cdf[-1].clone()
            rank = torch.searchsorted(cdf, u(n)).clamp_(max=nv - 1)
            mult = 2654435761 % nv | 1
            code = (rank * mult + int(float(u(1)) * nv)) % nv
            return (code * (2**32 // nv) - 2**31).to(torch.int32)
        if family == "gmix":
            k = 2 + int(10 * float(u(1)))
            means = -1.5e9 + 3e9 * u(k)
            sig = torch.exp(math.log(1e5) + (math.log(1e8) - math.log(1e5)) * u(k))
            wts = 0.5 + u(k)
            comp = torch.multinomial(wts / wts.sum(), n, replacement=True, generator=gen)
            x = means[comp] + sig[comp] * torch.randn(n, generator=gen, device=dev, dtype=torch.float64)
            return torch.round(x).clamp_(-2147483648.0, 2147483647.0).to(torch.int32)
        if family == "normal":
            sig = math.exp(math.log(1e4) + (math.log(1e9) - math.log(1e4)) * float(u(1)))
            x = sig * torch.randn(n, generator=gen, device=dev, dtype=torch.float64)
            return torch.round(x).clamp_(-2147483648.0, 2147483647.0).to(torch.int32)
        return torch.randint(-2**31, 2**31, (n,), generator=gen, device=dev, dtype=torch.int64).to(torch.int32)
    if family == "lognormal":
        sig = 0.5 + 2.5 * float(u(1))
        return torch.exp(sig * torch.randn(n, generator=gen, device=dev, dtype=torch.float64))
    if family == "gmix":
        k = 2 + int(10 * float(u(1)))
        means = -1e6 + 2e6 * u(k)
        sig = torch.exp(math.log(1e2) + (math.log(1e5) - math.log(1e2)) * u(k))
        comp = torch.multinomial(0.5 + u(k), n, replacement=True, generator=gen)
        return means[comp] + sig[comp] * torch.randn(n, generator=gen, device=dev, dtype=torch.float64)
    if family == "normal":
        return float(1 + 1e3 * float(u(1))) * torch.randn(n, generator=gen, device=dev, dtype=torch.float64)
    return -1e6 + 2e6 * u(n)


FAMILIES = {"i32": ("zipf", "gmix", "normal", "uniform"), "f64": ("lognormal", "gmix", "normal", "uniform")}


def positions(sample, v):
    """Positions in [0, 1023] of values v along the sorted sample (see module doc)."""
    torch = _torch()
    s = sample.to(torch.float64)
    vv = v.to(torch.float64)
    a = torch.searchsorted(s, vv, side="left")
    b = torch.searchsorted(s, vv, side="right")
    present = a < b
    lo = (a - 1).clamp(0, 1022)
    sl, sh = s[lo], s[lo + 1]
    frac = torch.where(sh > sl, (vv - sl) / (sh - sl), torch.zeros_like(vv)).clamp(0, 1)
    p = torch.where(present, (a + b - 1).to(torch.float64) / 2, lo.to(torch.float64) + frac)
    p = torch.where(vv < s[0], torch.zeros_like(p), p)
    p = torch.where(vv > s[-1], torch.full_like(p, 1023.0), p)
    return p


def pair(keys):
    """(sketch, target) of one array: the sketch from the unsorted keys, the
    targets from the keys the sort puts at ranks floor((j+1) n / 256)."""
    torch = _torch()
    x, _, sample = qs.sketch(keys)
    srt = keys.clone()
    qs.sort(srt)
    n = keys.numel()
    ranks = torch.tensor([((j + 1) * n) // 256 for j in range(NQ)], device=keys.device)
    t = positions(sample, srt[ranks]) / 1023.0
    return x, t.to(torch.float32)


def training_set(kind: str, count: int, n: int, seed: int):
    """count (sketch, target) pairs from arrays of n keys drawn from the kind's families."""
    torch = _torch()
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    xs, ts = [], []
    fams = FAMILIES[kind]
    for i in range(count):
        keys = draw_array(kind, fams[i % len(fams)], n, gen)
        x, t = pair(keys)
        xs.append(x)
        ts.append(t)
    return torch.stack(xs), torch.stack(ts)


# ---------------------------------------------------------------------------
# Model and training with the library's kernels.
# ---------------------------------------------------------------------------
def init_params(seed: int = 0):
    """He-scaled hidden layers, zero last layer: the untrained model outputs
    q_j = (j+1)/256 (the sampled splitters)."""
    torch = _torch()
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    p = torch.zeros(qs.mlp_param_count(), dtype=torch.float32, device="cuda")
    w1, b1 = 0, 64 * 1024
    w2, b2 = b1 + 64, b1 + 64 + 64 * 64
    p[w1:b1] = torch.randn(64 * 1024, generator=g, device="cuda") * math.sqrt(2.0 / 1024)
    p[b1:w2] = 0.01
    p[w2:b2] = torch.randn(64 * 64, generator=g, device="cuda") * math.sqrt(2.0 / 64)
    p[b2:b2 + 64] = 0.01
    return p


def train(X, T, steps: int = 1500, batch: int = 128, lr: float = 2e-3, seed: int = 0, params=None):
    """Adam on the mean squared quantile-position error; returns (params, losses)."""
    torch = _torch()
    p = init_params(seed) if params is None else params.clone()
    npar = p.numel()
    grad = torch.empty(npar, dtype=torch.float32, device="cuda")
    m = torch.zeros(npar, dtype=torch.float32, device="cuda")
    v = torch.zeros(npar, dtype=torch.float32, device="cuda")
    act = torch.empty(batch, 640, dtype=torch.float32, device="cuda")
    work = torch.empty(batch, 384, dtype=torch.float32, device="cuda")
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    g = torch.Generator(device="cuda")
    g.manual_seed(seed + 1)
    losses = []
    for step in range(1, steps + 1):
        idx = torch.randint(0, X.shape[0], (batch,), generator=g, device="cuda")
        xb = X[idx].contiguous()
        tb = T[idx].contiguous()
        qs.mlp_forward(p, xb, act)
        qs.mlp_backward(p, xb, tb, act, work, grad, loss)
        qs.mlp_adam(p, grad, m, v, step, lr)
        if step % 100 == 0 or step == steps:
            losses.append(float(loss.item()))
    return p, losses


def imbalance(keys, params=None) -> float:
    """Largest bucket / (n / 256) when `keys` (not modified) is cut by learned
    (params) or sampled (None) splitters: the balance the per-bucket sorts
    then see."""
    torch = _torch()
    work = keys.clone()
    qs.sort_learned(work, params)
    st = qs.stats()
    del work
    return st["bucket_max"] / (keys.numel() / 256.0)


def save(params, path: str) -> None:
    """Parameters as raw little-endian float32."""
    params.detach().cpu().numpy().astype("<f4").tofile(path)


def load_params(path: str):
    import numpy as np

    torch = _torch()
    return torch.from_numpy(np.fromfile(path, dtype="<f4")).to("cuda")
