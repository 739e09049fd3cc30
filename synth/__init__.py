"""Seeded synthetic COO tensors and factor matrices.

This module only draws random inputs; it holds none of the MTTKRP or CP-ALS
arithmetic.  Both the FP64 oracle and the CUDA path read the arrays it
returns, so the two sides always see identical inputs.

Every draw uses numpy's PCG64 generator from an explicit seed.  The workload
shapes stand in for the sparse tensors of the paper's evaluation (3- to
5-mode tensors, a short time-like mode, 3M-144M nonzeros), which are not
available here:

* ``plain``      3 modes 64x48x32, 4096 distinct uniform coordinates,
                 values U(0,1), R = 16, factors N(0,1).
* ``scale``      3 modes 1,000,000x500,000x200,000, each coordinate a
                 truncated Zipf(1.2) draw (inverse-CDF sampling), duplicates
                 removed keeping first occurrences, the first 50M kept,
                 values U(0,1), R = 32, factors N(0,1).
* ``precision``  4 modes 20,000x20,000x5,000x24, modes 0-2 Zipf(1.0), mode 3
                 uniform, 100M distinct coordinates, values lognormal(0,1),
                 R = 64.

* ``five``       5 modes 165,400 x 11,400 x 2 x 100 x 89 (the shape of the
                 paper's 5-mode tensor), modes 0-1 Zipf(1.1), the short modes
                 uniform, 26M distinct coordinates, values U(0,1), R = 32.
* ``batching``   512 independent 3-mode tensors, each dim log-uniform in
                 [100, 20,000], nnz log-uniform in [1e3, 2e6] (at most half
                 the cells, so that distinct coordinates can be drawn),
                 uniform coordinates, values U(0,1), R drawn from {16, 32}.
* ``serving``    a Poisson stream (mean 200 requests/s) of CP-ALS jobs, 3 or
                 4 modes, dims log-uniform in [1e3, 1e6], nnz log-uniform in
                 [1e4, 5e7], Zipf(1.1) coordinates, values U(0,1), R drawn
                 from {8, 16, 32, 64}.

A COO tensor is returned as ``(dims, idx, vals)`` with ``idx`` a list of
int32 arrays (one per mode) and ``vals`` float32.
"""
from __future__ import annotations

import numpy as np

PRESETS = {
    "plain": dict(dims=(64, 48, 32), nnz=4096, alphas=(None, None, None),
                  values="uniform", rank=16, seed=1),
    "scale": dict(dims=(1_000_000, 500_000, 200_000), nnz=50_000_000,
                  alphas=(1.2, 1.2, 1.2), values="uniform", rank=32, seed=2),
    "precision": dict(dims=(20_000, 20_000, 5_000, 24), nnz=100_000_000,
                      alphas=(1.0, 1.0, 1.0, None), values="lognormal",
                      rank=64, seed=3),
    "five": dict(dims=(165_400, 11_400, 2, 100, 89), nnz=26_000_000,
                 alphas=(1.1, 1.1, None, None, None), values="uniform", rank=32,
                 seed=6),
}


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


def zipf_cdf(n: int, alpha: float) -> np.ndarray:
    """Cumulative weights of k^-alpha, k = 1..n (unnormalised, float64)."""
    k = np.arange(1, n + 1, dtype=np.float64)
    return np.cumsum(k ** (-float(alpha)))


def draw_index(g: np.random.Generator, n: int, count: int,
               alpha: float | None, cdf: np.ndarray | None = None) -> np.ndarray:
    """`count` indices in [0, n): uniform when alpha is None, else truncated
    Zipf(alpha) on {1..n} by inverse-CDF sampling, shifted to start at 0."""
    if alpha is None:
        return g.integers(0, n, size=count, dtype=np.int64).astype(np.int32)
    if cdf is None:
        cdf = zipf_cdf(n, alpha)
    u = g.random(count) * cdf[-1]
    k = np.searchsorted(cdf, u, side="right")
    np.minimum(k, n - 1, out=k)
    return k.astype(np.int32)


def _linear(idx, dims):
    lin = np.zeros(idx[0].shape, dtype=np.int64)
    for c, n in zip(idx, dims):
        lin *= int(n)
        lin += c.astype(np.int64)
    return lin


def coo_distinct(dims, nnz, alphas=None, seed=0, values="uniform",
                 oversample=1.3):
    """COO tensor with `nnz` distinct coordinates.

    Coordinates are drawn mode by mode (uniform or truncated Zipf), repeated
    cells are dropped keeping their first occurrence, and the first `nnz`
    survivors in draw order are kept (more rounds are drawn if needed).
    Values: 'uniform' U(0,1) or 'lognormal' lognormal(0,1), float32."""
    dims = tuple(int(d) for d in dims)
    N = len(dims)
    alphas = tuple(alphas) if alphas is not None else (None,) * N
    cells = 1
    for d in dims:
        cells *= d
    if nnz > cells:
        raise ValueError("more nonzeros than cells")
    g = rng(seed)
    if all(a is None for a in alphas) and cells <= 4 * nnz + 1_000_000:
        lin = g.choice(cells, size=nnz, replace=False).astype(np.int64)
        idx = []
        for n in reversed(dims):
            idx.append((lin % n).astype(np.int32))
            lin //= n
        idx = idx[::-1]
    else:
        cdfs = [zipf_cdf(n, a) if a is not None else None
                for n, a in zip(dims, alphas)]
        kept = [np.empty(0, np.int32) for _ in dims]
        seen = np.empty(0, np.int64)
        need = nnz
        draw = int(nnz * oversample) + 1024
        while need > 0:
            cand = [draw_index(g, n, draw, a, c)
                    for n, a, c in zip(dims, alphas, cdfs)]
            lin = _linear(cand, dims)
            _, first = np.unique(lin, return_index=True)
            first.sort()
            fresh = first[~np.isin(lin[first], seen, assume_unique=False)] \
                if seen.size else first
            fresh = fresh[:need]
            for w in range(N):
                kept[w] = np.concatenate([kept[w], cand[w][fresh]])
            seen = np.concatenate([seen, lin[fresh]])
            need -= fresh.size
            draw = max(int(need * oversample * 2) + 1024, 4096)
        idx = kept
    if values == "uniform":
        vals = g.random(nnz, dtype=np.float32)
    elif values == "lognormal":
        vals = g.lognormal(0.0, 1.0, size=nnz).astype(np.float32)
    else:
        raise ValueError(values)
    return dims, [np.ascontiguousarray(c) for c in idx], vals


def coo_distinct_torch(dims, nnz, alphas=None, seed=0, values="uniform",
                       device="cpu", oversample=2.4, max_rounds=None):
    """The recipe of :func:`coo_distinct` drawn with torch on `device`.

    Used for the large workloads (tens of millions of nonzeros, where the
    Zipf heads make about half of all draws repeats): the draws are made in
    rounds on the device from a seeded torch generator, all draws so far are
    deduplicated together keeping first occurrences, and the first `nnz`
    survivors in draw order are kept.  The random stream differs from the
    numpy one, so the two functions give different (equally valid) tensors.
    With `max_rounds` the drawing stops after that many rounds and fewer
    than `nnz` nonzeros may be returned (heavily skewed small shapes).
    Returns (dims, idx list of int32 tensors, vals float32 tensor)."""
    import torch
    dims = tuple(int(d) for d in dims)
    N = len(dims)
    alphas = tuple(alphas) if alphas is not None else (None,) * N
    g = torch.Generator(device=device)
    g.manual_seed(int(seed))
    cdfs = []
    for n, a in zip(dims, alphas):
        if a is None:
            cdfs.append(None)
        else:
            k = torch.arange(1, n + 1, dtype=torch.float64, device=device)
            cdfs.append(torch.cumsum(k.pow(-float(a)), 0))
    strides = []
    s = 1
    for n in reversed(dims):
        strides.append(s)
        s *= n
    strides = strides[::-1]
    cand = [torch.empty(0, dtype=torch.int32, device=device) for _ in dims]
    draw = int(nnz * oversample) + 1024
    rounds = 0
    while True:
        rounds += 1
        for w, (n, c) in enumerate(zip(dims, cdfs)):
            if c is None:
                x = torch.randint(0, n, (draw,), generator=g, device=device,
                                  dtype=torch.int64)
            else:
                u = torch.rand(draw, generator=g, device=device,
                               dtype=torch.float64) * c[-1]
                x = torch.searchsorted(c, u, right=True).clamp_max_(n - 1)
            cand[w] = torch.cat([cand[w], x.to(torch.int32)])
        lin = torch.zeros(cand[0].numel(), dtype=torch.int64, device=device)
        for w in range(N):
            lin += cand[w].to(torch.int64) * strides[w]
        srt, order = torch.sort(lin, stable=True)
        head = torch.ones_like(srt, dtype=torch.bool)
        head[1:] = srt[1:] != srt[:-1]
        first = torch.sort(order[head]).values
        del lin, srt, order, head
        if first.numel() >= nnz:
            first = first[:nnz]
            break
        if max_rounds is not None and rounds >= max_rounds:
            nnz = int(first.numel())
            break
        draw = int((nnz - first.numel()) * oversample * 2) + 4096
    idx = [cand[w][first].contiguous() for w in range(N)]
    if values == "uniform":
        vals = torch.rand(nnz, generator=g, device=device, dtype=torch.float32)
    elif values == "lognormal":
        vals = torch.empty(nnz, device=device, dtype=torch.float32)
        vals.log_normal_(0.0, 1.0, generator=g)
    else:
        raise ValueError(values)
    return dims, idx, vals


def factors_torch(dims, rank, seed=0, device="cpu"):
    """Factor matrices I_w x R, N(0,1), float32 torch tensors on `device`."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(int(seed) + 1_000_003)
    return [torch.randn(int(n), int(rank), generator=g, device=device,
                        dtype=torch.float32) for n in dims]


def preset_torch(name: str, nnz: int | None = None, device="cpu"):
    """(dims, idx, vals, rank, factors) of a named workload as torch tensors
    drawn on `device` (see :func:`coo_distinct_torch`)."""
    p = PRESETS[name]
    n = p["nnz"] if nnz is None else int(nnz)
    dims, idx, vals = coo_distinct_torch(p["dims"], n, p["alphas"], p["seed"],
                                         p["values"], device)
    return dims, idx, vals, p["rank"], factors_torch(dims, p["rank"],
                                                     p["seed"], device)


def coo_random(dims, nnz, seed=0, duplicates=False):
    """Small COO tensor for tests: uniform coordinates, values U(0,1).
    With duplicates=True repeated coordinates are kept (they must sum)."""
    if not duplicates:
        return coo_distinct(dims, nnz, seed=seed)
    g = rng(seed)
    idx = [g.integers(0, int(n), size=nnz, dtype=np.int64).astype(np.int32)
           for n in dims]
    vals = g.random(nnz, dtype=np.float32)
    return tuple(int(d) for d in dims), idx, vals


def factors(dims, rank, seed=0):
    """Factor matrices I_w x R, N(0,1), float32, row-major."""
    g = rng(seed + 1_000_003)
    return [g.standard_normal((int(n), int(rank)), dtype=np.float32)
            for n in dims]


def preset(name: str, nnz: int | None = None):
    """(dims, idx, vals, rank, factors) of a named workload; `nnz` may shrink
    the tensor (the same recipe with fewer nonzeros) for quick runs."""
    p = PRESETS[name]
    n = p["nnz"] if nnz is None else int(nnz)
    dims, idx, vals = coo_distinct(p["dims"], n, p["alphas"], p["seed"],
                                   p["values"])
    return dims, idx, vals, p["rank"], factors(dims, p["rank"], p["seed"])


def rank_r_blocks(dims, rank, block, seed=0):
    """An exactly rank-R sparse tensor: component r lives on the index block
    [r*block, (r+1)*block) of every mode with positive entries a_r(i) > 0, so
    components never overlap and X = sum_r a_r o b_r o c_r exactly.
    Returns (dims, idx, vals(float64), true_factors)."""
    g = rng(seed)
    N = len(dims)
    for n in dims:
        if rank * block > n:
            raise ValueError("dims too small for the blocks")
    true = [np.zeros((int(n), rank)) for n in dims]
    for w in range(N):
        for r in range(rank):
            true[w][r * block:(r + 1) * block, r] = 0.5 + g.random(block)
    idx = [[] for _ in range(N)]
    vals = []
    grids = np.indices((block,) * N).reshape(N, -1).T
    for r in range(rank):
        for cell in grids:
            v = 1.0
            for w in range(N):
                i = r * block + int(cell[w])
                idx[w].append(i)
                v *= true[w][i, r]
            vals.append(v)
    idx = [np.asarray(a, dtype=np.int32) for a in idx]
    return tuple(int(d) for d in dims), idx, np.asarray(vals), true


def _log_uniform(g: np.random.Generator, lo: float, hi: float) -> float:
    return float(np.exp(g.uniform(np.log(lo), np.log(hi))))


def batching_specs(count: int = 512, seed: int = 4):
    """The batching workload: a list of (dims, nnz, rank, seed) per tensor."""
    g = rng(seed)
    out = []
    for t in range(count):
        dims = tuple(int(round(_log_uniform(g, 100, 20_000))) for _ in range(3))
        nnz = int(round(_log_uniform(g, 1e3, 2e6)))
        cells = int(np.prod(np.asarray(dims, dtype=np.float64)))
        nnz = max(1, min(nnz, cells // 2))
        rank = int(g.choice([16, 32]))
        out.append((dims, nnz, rank, seed * 1_000_000 + t))
    return out


def serving_specs(count: int, rate: float = 200.0, seed: int = 5):
    """The serving workload: a list of (arrival_s, dims, nnz, rank, seed)
    with Poisson arrivals of mean `rate` per second."""
    g = rng(seed)
    t = 0.0
    out = []
    for j in range(count):
        t += float(g.exponential(1.0 / rate))
        N = int(g.choice([3, 4]))
        dims = tuple(int(round(_log_uniform(g, 1e3, 1e6))) for _ in range(N))
        nnz = int(round(_log_uniform(g, 1e4, 5e7)))
        rank = int(g.choice([8, 16, 32, 64]))
        out.append((t, dims, nnz, rank, seed * 1_000_000 + j))
    return out


SERVING_ALPHA = 1.1


def tensor_torch(dims, nnz, seed, alpha=None, device="cpu", max_rounds=None):
    """One tensor of the batching (alpha None: uniform) or serving (Zipf
    alpha on every mode) workloads, drawn on `device`."""
    alphas = None if alpha is None else (alpha,) * len(dims)
    return coo_distinct_torch(dims, nnz, alphas, seed=seed, values="uniform",
                              device=device, max_rounds=max_rounds)
