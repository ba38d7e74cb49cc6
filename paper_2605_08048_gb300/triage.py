"""Learned triage for large batches of pair tests.

A small network (19 -> 256 -> 256 -> 9, BF16 weights, FP32 accumulation)
predicts, from cheap per-pair features (log n, log m, the 16 Ritz values of the
pooled scatter, T_obs), quantiles of the null distribution of |T| that the full
permutation test would draw.  From them a predicted p follows; pairs whose
predicted p lies clearly outside a band around alpha are decided without the
full test, every pair inside the band and a random audit sample get the full
test, and the audit measures the network's decision error.

The network is trained by the library's own kernels (forward, backward,
pinball loss, Adam) on targets produced by the library's own full tests of
training pairs (empirical quantiles of |T_b|).  This module only orchestrates
those calls; all arithmetic runs on the GPU.
"""
from __future__ import annotations

import time
from dataclasses import dataclass, field

import numpy as np
import torch

from . import hbperm as H


def init_params(seed: int = 0, device="cuda") -> torch.Tensor:
    """He-normal weights and zero biases in the flat layout of the network."""
    rng = np.random.default_rng(seed)
    parts = []
    for fan_in, fan_out in ((H.TRIAGE_NFEAT, 256), (256, 256), (256, H.TRIAGE_NQ)):
        parts.append(rng.standard_normal((fan_in, fan_out)) * np.sqrt(2.0 / fan_in))
        parts.append(np.zeros(fan_out))
    flat = np.concatenate([p.ravel() for p in parts]).astype(np.float32)
    assert flat.size == H.mlp_param_count()
    return torch.from_numpy(flat).to(device)


def _dev_bf16(xy_bits: np.ndarray) -> torch.Tensor:
    return torch.from_numpy(np.ascontiguousarray(xy_bits).view(np.int16)).view(torch.bfloat16).cuda()


def training_set(ctx: H.Context, batches, opts: H.hb_opts):
    """Features and null-quantile targets of the pairs of each synthetic batch."""
    feats, targets = [], []
    for b in batches:
        XY = _dev_bf16(b.XY) if b.XY.dtype == np.uint16 else torch.from_numpy(b.XY).cuda()
        f, _, r1 = H.triage_features(ctx, XY, b.n, b.m, opts)
        q, r2 = H.null_quantiles(ctx, XY, b.n, b.m, opts)
        ok = torch.tensor([a["status"] == 0 and c["status"] == 0 for a, c in zip(r1, r2)], device=f.device)
        feats.append(f[ok])
        targets.append(q[ok])
    return torch.cat(feats), torch.cat(targets)


def train(ctx: H.Context, feat: torch.Tensor, target: torch.Tensor, epochs: int = 60, batch: int = 1024,
          lr: float = 1e-3, seed: int = 0):
    """Adam on the mean pinball loss; returns (network, per-epoch mean loss)."""
    net = H.MLP(init_params(seed, feat.device))
    g = torch.Generator(device="cpu").manual_seed(seed)
    P = feat.shape[0]
    history = []
    for _ in range(epochs):
        perm = torch.randperm(P, generator=g).to(feat.device)
        losses = []
        for s in range(0, P, batch):
            idx = perm[s:s + batch]
            if idx.numel() < 2:
                continue
            losses.append(net.grad_step(ctx, feat[idx].contiguous(), target[idx].contiguous()))
            net.adam(lr)
        history.append(float(torch.stack(losses).mean()))
    return net, history


@dataclass
class TriageReport:
    pairs: int
    full_tested: int
    audited: int
    skipped: int
    audit_decision_error: float
    decision_error_skipped: float      # against full tests of every skipped pair (evaluation only)
    seconds_features: float
    seconds_full_subset: float
    seconds_full_all: float
    p_hat: np.ndarray = field(repr=False, default=None)
    p_full: np.ndarray = field(repr=False, default=None)


def triage(ctx: H.Context, net: H.MLP, batch, opts: H.hb_opts, alpha: float = 0.05, band=(0.005, 0.2),
           audit: float = 0.02, seed: int = 0, evaluate_all: bool = True) -> TriageReport:
    """Routes the pairs of `batch`: full test for predicted p in `band` and for
    an audit sample; the others are decided by the predicted p."""
    XY = _dev_bf16(batch.XY) if batch.XY.dtype == np.uint16 else torch.from_numpy(batch.XY).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    feat, tobs, res = H.triage_features(ctx, XY, batch.n, batch.m, opts)
    q = net.forward(ctx, feat)
    p_hat = H.triage_predict_p(q, tobs).cpu().numpy()
    torch.cuda.synchronize()
    t_feat = time.perf_counter() - t0
    P = len(batch.n)
    rng = np.random.default_rng(seed)
    in_band = (p_hat >= band[0]) & (p_hat <= band[1])
    audit_mask = (~in_band) & (rng.random(P) < audit)
    full = in_band | audit_mask
    sub = np.nonzero(full)[0]
    t_sub = 0.0
    p_full = np.full(P, np.nan)
    if len(sub):
        b2 = _subset(batch, sub)
        X2 = _dev_bf16(b2.XY) if b2.XY.dtype == np.uint16 else torch.from_numpy(b2.XY).cuda()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = H.hb_perm_test_batched(ctx, X2, b2.n, b2.m, opts)
        t_sub = time.perf_counter() - t0
        p_full[sub] = [x["p"] for x in r]
    t_all = float("nan")
    if evaluate_all:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = H.hb_perm_test_batched(ctx, XY, batch.n, batch.m, opts)
        t_all = time.perf_counter() - t0
        p_all = np.array([x["p"] for x in r])
    dec_hat = p_hat <= alpha
    a = np.nonzero(audit_mask)[0]
    audit_err = float(np.mean(dec_hat[a] != (p_full[a] <= alpha))) if len(a) else float("nan")
    skipped = np.nonzero(~in_band)[0]
    err_skipped = float(np.mean(dec_hat[skipped] != (p_all[skipped] <= alpha))) if evaluate_all and len(skipped) \
        else float("nan")
    return TriageReport(P, int(full.sum()), int(audit_mask.sum()), int((~full).sum()), audit_err, err_skipped,
                        t_feat, t_sub, t_all, p_hat, p_all if evaluate_all else p_full)


def _subset(batch, idx):
    from .synth import Batch

    off = batch.offsets
    rows = np.concatenate([np.arange(off[p], off[p + 1]) for p in idx])
    return Batch(batch.XY[rows], batch.n[idx], batch.m[idx], batch.d, batch.dtype, batch.null[idx])
