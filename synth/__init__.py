"""Seeded synthetic workloads shaped like the paper's (Sec. 5.1, Sec. 5.3).

This module only draws inputs; it holds none of the index or search
arithmetic, and both the oracle side and the CUDA side consume the bytes it
writes.

* Random walks (Sec. 5.1): x_0 ~ N(0,1), x_t = x_{t-1} + N(0,1), then each
  series is z-normalised (mean 0, population standard deviation 1).
* Fresh queries: random walks drawn from a separate seed.
* Noisy members (Sec. 5.3, "query workloads of increasing difficulty"): a
  dataset series chosen at random plus N(0, sigma) noise on every point, not
  re-normalised.

Two back ends draw the same recipe: numpy on the host (small cases, CPU
tests) and torch on a CUDA device (full-size collections, chunked so peak
memory stays at the output size).  They do not produce the same numbers;
whichever bytes were drawn are the dataset.
"""
from __future__ import annotations

import numpy as np

DATASET_SEED = 1234
QUERY_SEED = 5678
NOISE_SEED = 91011


def _znorm_np(x: np.ndarray) -> np.ndarray:
    mu = x.mean(axis=1, keepdims=True)
    sd = x.std(axis=1, keepdims=True)          # population std (divide by n)
    sd[sd == 0] = 1.0
    return (x - mu) / sd


def random_walks(N: int, n: int, seed: int = DATASET_SEED, znorm: bool = True) -> np.ndarray:
    """N random-walk series of length n as float32 [N, n] (numpy, host)."""
    rng = np.random.default_rng(seed)
    out = np.empty((N, n), dtype=np.float32)
    step = 1 << 16
    for lo in range(0, N, step):
        hi = min(N, lo + step)
        x = np.cumsum(rng.standard_normal((hi - lo, n)), axis=1)
        out[lo:hi] = _znorm_np(x) if znorm else x
    return out


def noisy_members(data: np.ndarray, count: int, sigma: float, seed: int = NOISE_SEED):
    """(queries, member_ids): random dataset rows plus N(0, sigma) noise."""
    rng = np.random.default_rng(seed)
    ids = rng.integers(0, data.shape[0], size=count)
    q = data[ids].astype(np.float64) + rng.normal(0.0, sigma, size=(count, data.shape[1]))
    return q.astype(np.float32), ids


def query_mix(data: np.ndarray, count: int, sigmas=(0.1, 0.5, 1.0), seed: int = QUERY_SEED):
    """Half fresh random walks, half noisy members split evenly over sigmas."""
    n = data.shape[1]
    n_fresh = count // 2
    parts = [random_walks(n_fresh, n, seed=seed)]
    rest = count - n_fresh
    for i, s in enumerate(sigmas):
        c = rest // len(sigmas) + (1 if i < rest % len(sigmas) else 0)
        if c:
            parts.append(noisy_members(data, c, s, seed=NOISE_SEED + i)[0])
    return np.concatenate(parts, axis=0)


# ----------------------------------------------------------- torch / device
def random_walks_torch(N: int, n: int, seed: int = DATASET_SEED, device="cuda",
                       chunk: int = 1 << 20, out=None):
    """N random-walk series of length n as a float32 torch tensor on ``device``."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(seed)
    if out is None:
        out = torch.empty((N, n), dtype=torch.float32, device=device)
    for lo in range(0, N, chunk):
        hi = min(N, lo + chunk)
        x = torch.randn((hi - lo, n), generator=g, device=device, dtype=torch.float32)
        torch.cumsum(x, dim=1, out=x)
        mu = x.mean(dim=1, keepdim=True)
        sd = x.std(dim=1, keepdim=True, unbiased=False)
        sd = torch.where(sd == 0, torch.ones_like(sd), sd)
        out[lo:hi] = (x - mu) / sd
        del x
    return out


def noisy_members_torch(data, count: int, sigma: float, seed: int = NOISE_SEED):
    import torch

    g = torch.Generator(device=data.device)
    g.manual_seed(seed)
    ids = torch.randint(0, data.shape[0], (count,), generator=g, device=data.device)
    noise = torch.randn((count, data.shape[1]), generator=g, device=data.device) * sigma
    return (data[ids] + noise).contiguous(), ids


def query_mix_torch(data, count: int, sigmas=(0.1, 0.5, 1.0), seed: int = QUERY_SEED):
    import torch

    n = data.shape[1]
    n_fresh = count // 2
    parts = [random_walks_torch(n_fresh, n, seed=seed, device=data.device)] if n_fresh else []
    rest = count - n_fresh
    for i, s in enumerate(sigmas):
        c = rest // len(sigmas) + (1 if i < rest % len(sigmas) else 0)
        if c:
            parts.append(noisy_members_torch(data, c, s, seed=NOISE_SEED + i)[0])
    return torch.cat(parts, dim=0).contiguous()
