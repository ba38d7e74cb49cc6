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


def _dev_bf16(xy) -> torch.Tensor:
    """The batch's rows on the device (BF16 bit patterns from numpy, or a tensor as is)."""
    if isinstance(xy, torch.Tensor):
        return xy if xy.is_cuda else xy.cuda()
    return torch.from_numpy(np.ascontiguousarray(xy).view(np.int16)).view(torch.bfloat16).cuda()


def _on_device(b) -> torch.Tensor:
    if isinstance(b.XY, torch.Tensor) or b.XY.dtype == np.uint16:
        return _dev_bf16(b.XY)
    return torch.from_numpy(b.XY).cuda()


def training_set(ctx: H.Context, batches, opts: H.hb_opts):
    """Features and null-quantile targets of the pairs of each synthetic batch."""
    feats, targets = [], []
    for b in batches:
        XY = _on_device(b)
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
    XY = _on_device(batch)
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
        # gathering the routed pairs into their own packed batch is part of the triage's cost
        t0 = time.perf_counter()
        p_full[sub] = test_subset(ctx, XY, batch.n, batch.m, sub, opts)
        t_sub = time.perf_counter() - t0
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


def test_subset(ctx: H.Context, XY: torch.Tensor, n, m, idx, opts: H.hb_opts) -> np.ndarray:
    """The full test (hb_perm_test_batched) of the pairs `idx` of a packed
    device batch, gathered into a packed batch of their own; their p-values."""
    X2, n2, m2 = pack(XY, n, m, idx)
    r = H.hb_perm_test_batched(ctx, X2, n2, m2, opts)
    return np.array([x["p"] for x in r])


def pack(XY: torch.Tensor, n, m, idx):
    """The pairs `idx` of a packed device batch as a new packed batch."""
    from .shard import pack as _pack

    return _pack(XY, n, m, np.asarray(idx))


def evaluate_at_scale(ctx: H.Context, train_pairs: int = 200_000, eval_pairs: int = 50_000, chunk: int = 4096,
                      opts: H.hb_opts = None, epochs: int = 30, lr: float = 2e-3, alpha: float = 0.05,
                      band=(0.005, 0.2), audit: float = 0.02, seed: int = 0, log=None) -> dict:
    """Trains the network on the method's own runs of `train_pairs` synthetic
    pairs of the batched recipe, then triages `eval_pairs` held-out pairs in
    chunks of `chunk`, testing every pair fully as well to measure the
    decision error and the time the triage saves.  Returns the totals."""
    from . import synth

    opts = opts or H.make_opts(B=9999, seed=1, path=H.HB_PATH_MIXED_2SM)
    say = log or (lambda *_: None)
    t0 = time.perf_counter()
    feats, targets = [], []
    for k, c0 in enumerate(range(0, train_pairs, chunk)):
        b = synth.batch_device(100_000 + k, min(chunk, train_pairs - c0))
        f, q = training_set(ctx, [b], opts)
        feats.append(f)
        targets.append(q)
        del b
    feat, target = torch.cat(feats), torch.cat(targets)
    t_data = time.perf_counter() - t0
    say(f"training set: {feat.shape[0]} pairs in {t_data:.1f} s")
    t0 = time.perf_counter()
    net, hist = train(ctx, feat, target, epochs=epochs, batch=1024, lr=lr, seed=seed)
    t_train = time.perf_counter() - t0
    say(f"training: loss {hist[0]:.4f} -> {hist[-1]:.4f} in {t_train:.1f} s")
    warm = synth.batch_device(199_999, 256)
    triage(ctx, net, warm, opts, alpha, band, audit, seed=seed)  # workspace sizing
    tot = dict(pairs=0, skipped=0, full_tested=0, audited=0, audit_wrong=0, skipped_wrong=0, seconds_features=0.0,
               seconds_full_subset=0.0, seconds_full_all=0.0)
    for k, c0 in enumerate(range(0, eval_pairs, chunk)):
        b = synth.batch_device(200_000 + k, min(chunk, eval_pairs - c0))
        r = triage(ctx, net, b, opts, alpha, band, audit, seed=seed + k)
        tot["pairs"] += r.pairs
        tot["skipped"] += r.skipped
        tot["full_tested"] += r.full_tested
        tot["audited"] += r.audited
        tot["audit_wrong"] += int(round(r.audit_decision_error * r.audited)) if r.audited else 0
        tot["skipped_wrong"] += int(round(r.decision_error_skipped * r.skipped)) if r.skipped else 0
        tot["seconds_features"] += r.seconds_features
        tot["seconds_full_subset"] += r.seconds_full_subset
        tot["seconds_full_all"] += r.seconds_full_all
        del b
    tot.update(train_pairs=int(feat.shape[0]), epochs=epochs, loss_first=hist[0], loss_last=hist[-1],
               seconds_training_data=t_data, seconds_training=t_train,
               decision_error_skipped=tot["skipped_wrong"] / max(1, tot["skipped"]),
               audit_decision_error=tot["audit_wrong"] / max(1, tot["audited"]),
               skipped_fraction=tot["skipped"] / max(1, tot["pairs"]),
               speedup=tot["seconds_full_all"] / max(1e-9, tot["seconds_features"] + tot["seconds_full_subset"]))
    return tot
