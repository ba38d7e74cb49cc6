"""Seeded synthetic token-embedding clouds.

This module only draws inputs; it holds none of the test's arithmetic.  Each
row is ``normalize(mu_g + sigma_g * N(0, I_d))`` with ``mu_g`` a unit mean
direction, which mimics an l2-normalised contextual-embedding cloud (the
paper's Sec. 3.1 normalisation step).  The paper's corpora and language models
are not available, so these clouds stand in for them with the shapes of its
workloads (d = 768 for base-size encoders, d = 1024 for large ones).

Generation uses numpy's PCG64 with seeds derived from ``SeedSequence`` so the
same seed gives the same bits on every platform.  BF16 data are returned as
``uint16`` bit patterns (round-to-nearest-even from FP32).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
from dataclasses import dataclass

import numpy as np


def to_bf16_bits(a: np.ndarray) -> np.ndarray:
    """FP32 -> BF16 bit patterns, round-to-nearest-even (finite inputs)."""
    bits = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32)
    bias = ((bits >> 16) & 1) + np.uint32(0x7FFF)
    return ((bits + bias) >> 16).astype(np.uint16)


def bf16_bits_to_f32(b: np.ndarray) -> np.ndarray:
    return (np.asarray(b, dtype=np.uint16).astype(np.uint32) << 16).view(np.float32)


def _rng(seed: int, *key: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed) & 0xFFFFFFFF, *map(int, key)])))


def unit(rng: np.random.Generator, d: int) -> np.ndarray:
    v = rng.standard_normal(d)
    return v / np.linalg.norm(v)


def cloud(rng: np.random.Generator, mu: np.ndarray, sigma: float, rows: int, dtype: str = "f32") -> np.ndarray:
    d = mu.shape[0]
    x = rng.standard_normal((rows, d), dtype=np.float32).astype(np.float64)
    x *= sigma
    x += mu
    x /= np.linalg.norm(x, axis=1, keepdims=True)
    x32 = x.astype(np.float32)
    return to_bf16_bits(x32) if dtype == "bf16" else x32


def pair(seed: int, n: int, m: int, d: int, sigma_x: float = 0.35, sigma_y: float = 0.35, angle_deg=None,
         dtype: str = "f32", key: int = 0):
    """One (X, Y) pair.  With ``angle_deg`` the mean directions are at that
    angle; otherwise they are independent random unit vectors."""
    rng = _rng(seed, key)
    mx = unit(rng, d)
    if angle_deg is None:
        my = unit(rng, d)
    else:
        w = rng.standard_normal(d)
        w -= (w @ mx) * mx
        w /= np.linalg.norm(w)
        t = np.deg2rad(angle_deg)
        my = np.cos(t) * mx + np.sin(t) * w
    X = cloud(rng, mx, sigma_x, n, dtype)
    Y = cloud(rng, my, sigma_y, m, dtype)
    return X, Y


def lognormal_sizes(seed: int, P: int, median: float = 300.0, sigma_log: float = 1.0, lo: int = 20, hi: int = 8000):
    rng = _rng(seed, 0xC0FFEE)
    z = rng.standard_normal((P, 2))
    s = np.clip(np.rint(np.exp(np.log(median) + sigma_log * z)), lo, hi).astype(np.int64)
    return s[:, 0].copy(), s[:, 1].copy()


@dataclass
class Batch:
    XY: np.ndarray        # [sum(n+m)][d] packed: pair p = n[p] rows of X then m[p] rows of Y
    n: np.ndarray
    m: np.ndarray
    d: int
    dtype: str
    null: np.ndarray      # bool per pair: True = equal dispersion

    @property
    def offsets(self):
        o = np.zeros(len(self.n) + 1, dtype=np.int64)
        np.cumsum(self.n + self.m, out=o[1:])
        return o

    def pair(self, p: int):
        o = self.offsets
        a = self.XY[o[p]:o[p] + self.n[p]]
        b = self.XY[o[p] + self.n[p]:o[p + 1]]
        return a, b


def batch(seed: int, P: int, d: int = 768, dtype: str = "bf16", sizes=None, sigma: float = 0.35,
          alt_ratio: float = 1.1, threads: int | None = None) -> Batch:
    """Batched workload: lognormal sizes (median 300, sigma_log 1, clipped
    20..8000); the first half of the pairs are null (equal sigma, random
    directions), the second half alternatives (sigma_X = alt_ratio * sigma)."""
    n, m = sizes if sizes is not None else lognormal_sizes(seed, P)
    n = np.asarray(n, dtype=np.int64)
    m = np.asarray(m, dtype=np.int64)
    null = np.arange(P) < (P + 1) // 2
    off = np.zeros(P + 1, dtype=np.int64)
    np.cumsum(n + m, out=off[1:])
    XY = np.empty((int(off[-1]), d), dtype=np.uint16 if dtype == "bf16" else np.float32)

    def fill(p):
        sx = sigma if null[p] else sigma * alt_ratio
        X, Y = pair(seed, int(n[p]), int(m[p]), d, sx, sigma, None, dtype, key=p + 1)
        XY[off[p]:off[p] + n[p]] = X
        XY[off[p] + n[p]:off[p + 1]] = Y

    workers = threads or min(32, os.cpu_count() or 1)
    with cf.ThreadPoolExecutor(workers) as ex:
        list(ex.map(fill, range(P)))
    return Batch(XY, n, m, d, dtype, null)


def batch_device(seed: int, P: int, d: int = 768, sigma: float = 0.35, alt_ratio: float = 1.1, device="cuda",
                 null_fraction: float = 0.5) -> Batch:
    """The batched recipe generated on the GPU (for batches too large to draw
    on the host): the same lognormal sizes and cloud model as `batch`, rows =
    normalize(mu + sigma N(0, I)) rounded to BF16, with torch's device
    generator seeded by `seed` (a different random stream from `batch`'s).
    The first null_fraction of the pairs are null, the rest alternatives
    (sigma_X = alt_ratio * sigma).  XY is a BF16 CUDA tensor."""
    import torch

    n, m = lognormal_sizes(seed, P)
    n = np.asarray(n, dtype=np.int64)
    m = np.asarray(m, dtype=np.int64)
    null = np.arange(P) < int(round(null_fraction * P))
    g = torch.Generator(device=device).manual_seed(int(seed))
    mu = torch.randn((2 * P, d), generator=g, device=device)
    mu /= mu.norm(dim=1, keepdim=True)                     # pair p: rows 2p (X), 2p+1 (Y)
    sig = torch.tensor(np.stack([np.where(null, sigma, sigma * alt_ratio), np.full(P, sigma)], 1).reshape(-1),
                       dtype=torch.float32, device=device)
    sizes = torch.from_numpy(np.stack([n, m], 1).reshape(-1)).to(device)
    owner = torch.repeat_interleave(torch.arange(2 * P, device=device), sizes)
    XY = torch.empty((int(sizes.sum()), d), dtype=torch.bfloat16, device=device)
    step = 1 << 18
    for r0 in range(0, XY.shape[0], step):                 # bounded FP32 scratch
        o = owner[r0:r0 + step]
        x = torch.randn((o.numel(), d), generator=g, device=device) * sig[o, None] + mu[o]
        XY[r0:r0 + step] = (x / x.norm(dim=1, keepdim=True)).to(torch.bfloat16)
    return Batch(XY, n, m, d, "bf16", null)


# Workload recipes (sizes and distributions of the paper's workloads).
def workload_plain(seed: int = 1235):
    """Single test: n=200, m=300, d=768, FP32, sigma 0.35 both, independent
    random mean directions (null: equal breadth, different directions)."""
    return pair(seed, 200, 300, 768, 0.35, 0.35, None, "f32")


def workload_large(seed: int = 1236):
    """Large single pair: n=m=5000, d=1024, BF16; sigma_X 0.35, sigma_Y 0.40."""
    return pair(seed, 5000, 5000, 1024, 0.35, 0.40, None, "bf16")


def workload_batched(seed: int = 1237, P: int = 4096):
    """4096 pairs, lognormal sizes, d=768 BF16, half null, half alternative."""
    return batch(seed, P, 768, "bf16")


def workload_calibration(seed: int = 1238, pairs_per_angle: int = 200, n: int = 500, d: int = 768,
                         dtype: str = "bf16", angles=None):
    """Type-I sweep: equal sigma 0.35, mean-direction angle 0..90 degrees."""
    angles = list(np.linspace(0.0, 90.0, 10)) if angles is None else list(angles)
    out = []
    for a_idx, a in enumerate(angles):
        for k in range(pairs_per_angle):
            X, Y = pair(seed, n, n, d, 0.35, 0.35, a, dtype, key=1000 * a_idx + k)
            out.append((a, X, Y))
    return out
