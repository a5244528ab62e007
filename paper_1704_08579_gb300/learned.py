"""Training and evaluation of the splitter MLP (learned form of the sort).

The network is trained on (sketch, exact quantile) pairs that the sort itself
generates: for each training array the library computes the 1024-key sketch
(qs_sketch_*) and sorts the array (qs_sort_*); the targets are the keys at
ranks floor((j+1) n / 256), j = 0..254, of the sorted array, expressed as
positions along the curve the sort reads the model's output on -- the sorted
sample smoothed by a 17-key centred moving average (a key between two curve
points maps to the linear interpolation between their positions, a key equal
to a run of curve points to the run's middle).  The
forward, backward and Adam steps are the library's own kernels
(qs_mlp_forward / qs_mlp_backward / qs_mlp_adam); torch only holds buffers and
draws the training arrays.

The untrained network (last layer zero) outputs q_j = (j+1)/256: evenly
spaced positions on the curve; training moves it from there.
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


CURVE_HALF = 8  # moving-average half window of the curve the positions are read on


def curve(sample):
    """The sorted sample smoothed by a centred moving average over 17 keys,
    the window shrinking symmetrically at both ends (float64)."""
    torch = _torch()
    s = sample.to(torch.float64)
    m = s.numel()
    c = torch.cat([torch.zeros(1, dtype=torch.float64, device=s.device), torch.cumsum(s, 0)])
    i = torch.arange(m, device=s.device)
    h = torch.minimum(torch.minimum(i, m - 1 - i), torch.full_like(i, CURVE_HALF))
    return (c[i + h + 1] - c[i - h]) / (2 * h + 1).to(torch.float64)


def positions(cv, v):
    """Positions in [0, 1023] of values v along the non-decreasing curve cv
    (the middle of a run of equal curve points, else linear interpolation)."""
    torch = _torch()
    vv = v.to(torch.float64)
    a = torch.searchsorted(cv, vv, side="left")
    b = torch.searchsorted(cv, vv, side="right")
    present = a < b
    lo = (a - 1).clamp(0, cv.numel() - 2)
    sl, sh = cv[lo], cv[lo + 1]
    frac = torch.where(sh > sl, (vv - sl) / (sh - sl), torch.zeros_like(vv)).clamp(0, 1)
    p = torch.where(present, (a + b - 1).to(torch.float64) / 2, lo.to(torch.float64) + frac)
    p = torch.where(vv < cv[0], torch.zeros_like(p), p)
    p = torch.where(vv > cv[-1], torch.full_like(p, cv.numel() - 1.0), p)
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
    t = positions(curve(sample), srt[ranks]) / 1023.0
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


def imbalance(keys, params=None) -> dict:
    """Bucket balance when `keys` (not modified) is cut by learned (params) or
    sampled (None) splitters, as the bucket pass of the sort reports it:
    err = total variation distance between the bucket sizes and an even split
    (0 = perfect), max = largest bucket / even share, over = buckets above the
    fallback bound."""
    work = keys.clone()
    qs.sort_learned(work, params)
    st = qs.stats()
    del work
    n = keys.numel()
    return {"err": st["bucket_dev"] / (2.0 * n * 256), "max": st["bucket_max"] / (n / 256.0), "over": st["bucket_over"]}


def position_error(params, X, T) -> float:
    """Mean squared error of the model's positions against the targets."""
    q = qs.mlp_forward(params, X)
    return float(((q - T) ** 2).mean().item())


def compare(params, kind: str, count: int, n: int, seed: int) -> dict:
    """Mean bucket-imbalance error per family on fresh arrays: the trained
    model (params), the untrained one (even positions on the curve) and the
    sampled splitters (every 4th sample key)."""
    torch = _torch()
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    init = init_params(0)
    fams = FAMILIES[kind]
    out = {f: {"learned": [], "untrained": [], "sampled": []} for f in fams}
    for i in range(count):
        f = fams[i % len(fams)]
        keys = draw_array(kind, f, n, gen)
        out[f]["learned"].append(imbalance(keys, params)["err"])
        out[f]["untrained"].append(imbalance(keys, init)["err"])
        out[f]["sampled"].append(imbalance(keys, None)["err"])
    return {f: {k: sum(v) / len(v) for k, v in d.items()} for f, d in out.items()}


def save(params, path: str) -> None:
    """Parameters as raw little-endian float32."""
    params.detach().cpu().numpy().astype("<f4").tofile(path)


def load_params(path: str):
    import numpy as np

    torch = _torch()
    return torch.from_numpy(np.fromfile(path, dtype="<f4")).to("cuda")
