"""FP64 numpy oracle of the learned-triage pieces.

TEST INFRASTRUCTURE ONLY: the test-suite and the smoke check may import this
module; the product path never does.  It shares no code with the CUDA
kernels.  The paper has no learned component; these definitions are the
library's triage model, written out plainly:

- features: log n, log m, log(d * lambda_k) for the 16 Ritz values lambda_k of
  the pooled scatter Z^T Z / N after a fixed number of block subspace
  iterations from a fixed start block, and 10 * T_obs (19 values);
- MLP 19 -> 256 -> 256 -> 9 with ReLU, weights rounded to BF16, FP32 biases;
- pinball (quantile) loss against the empirical null quantiles of |T_b|;
- Adam (Kingma and Ba, 2015);
- predicted p from the predicted quantiles by linear interpolation.
"""
from __future__ import annotations

import math

import numpy as np

from . import oracle as O

K_RITZ = 16
RITZ_ITERS = 2
LEVELS = np.array([0.5, 0.8, 0.9, 0.95, 0.975, 0.99, 0.995, 0.998, 0.999])
N_FEAT = 19
HIDDEN = 256
N_OUT = 9
TARGET_SCALE = 100.0


def start_block(d: int, k: int = K_RITZ) -> np.ndarray:
    """Fixed start block: entry (j, c) = (w >> 8) / 2^24 - 1/2 with w the first
    Philox4x32-10 word of counter (j, c, 0x5EED, 0) under key (0, 0)."""
    V = np.zeros((d, k), dtype=np.float64)
    for j in range(d):
        for c in range(k):
            w = int(O.philox4x32_10([j, c, 0x5EED, 0], [0, 0])[0])
            V[j, c] = (w >> 8) / float(1 << 24) - 0.5
    return V


def mgs(W: np.ndarray) -> np.ndarray:
    """Modified Gram-Schmidt on the columns, in column order."""
    V = W.astype(np.float64).copy()
    for c in range(V.shape[1]):
        for l in range(c):
            V[:, c] -= (V[:, l] @ V[:, c]) * V[:, l]
        V[:, c] /= np.linalg.norm(V[:, c])
    return V


def ritz_values(Z: np.ndarray, iters: int = RITZ_ITERS, V0=None) -> np.ndarray:
    """Ritz values (descending) of S = Z^T Z / N on the block after `iters`
    steps V <- orth(S V) from V0."""
    Z = np.asarray(Z, dtype=np.float64)
    N, d = Z.shape
    V = mgs(start_block(d) if V0 is None else V0)
    for _ in range(iters):
        V = mgs(Z.T @ (Z @ V) / N)
    H = V.T @ (Z.T @ (Z @ V)) / N
    H = 0.5 * (H + H.T)
    return np.sort(np.linalg.eigvalsh(H))[::-1]


def features(X: np.ndarray, Y: np.ndarray, T_obs: float, align: int = 1) -> np.ndarray:
    st, Z, _, _, _ = O.align(X, Y, align=align)
    assert st == O.OK
    from paper_2605_08048_gb300 import synth  # input decoding only

    z = synth.bf16_bits_to_f32(Z).astype(np.float64) if Z.dtype == np.uint16 else Z.astype(np.float64)
    lam = ritz_values(z)
    d = z.shape[1]
    f = np.empty(N_FEAT)
    f[0] = math.log(X.shape[0])
    f[1] = math.log(Y.shape[0])
    f[2:18] = np.log(np.maximum(lam * d, 1e-12))
    f[18] = 10.0 * T_obs
    return f


def param_layout():
    """Flat parameter vector: W1[19][256], b1, W2[256][256], b2, W3[256][9], b3."""
    shapes = [(N_FEAT, HIDDEN), (HIDDEN,), (HIDDEN, HIDDEN), (HIDDEN,), (HIDDEN, N_OUT), (N_OUT,)]
    offs, o = [], 0
    for s in shapes:
        offs.append(o)
        o += int(np.prod(s))
    return shapes, offs, o


def unpack(params: np.ndarray):
    shapes, offs, _ = param_layout()
    return [params[o:o + int(np.prod(s))].reshape(s) for s, o in zip(shapes, offs)]


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round to FP32, then to BF16 nearest-even (finite values), as float64:
    keep the top 16 bits of the FP32 pattern after adding 0x7FFF plus the
    lowest kept bit (ties go to the even pattern)."""
    u = np.ascontiguousarray(np.asarray(a, dtype=np.float32)).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)
    return r.view(np.float32).astype(np.float64)


def mlp_forward(params: np.ndarray, F: np.ndarray):
    W1, b1, W2, b2, W3, b3 = unpack(params)
    W1, W2, W3 = bf16_round(W1), bf16_round(W2), bf16_round(W3)
    b1, b2, b3 = (np.asarray(v, dtype=np.float32).astype(np.float64) for v in (b1, b2, b3))
    a1 = F @ W1 + b1
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ W2 + b2
    h2 = np.maximum(a2, 0.0)
    y = h2 @ W3 + b3
    return y, (F, a1, h1, a2, h2)


def mlp_backward(params: np.ndarray, cache, dy: np.ndarray) -> np.ndarray:
    """Gradient of sum(dy * y) with respect to the flat parameters (the
    weights enter the forward rounded to BF16; the gradient is taken with
    respect to those rounded values, straight through the rounding)."""
    W1, b1, W2, b2, W3, b3 = unpack(params)
    W2r, W3r = bf16_round(W2), bf16_round(W3)
    F, a1, h1, a2, h2 = cache
    gW3 = h2.T @ dy
    gb3 = dy.sum(0)
    dh2 = dy @ W3r.T
    da2 = dh2 * (a2 > 0)
    gW2 = h1.T @ da2
    gb2 = da2.sum(0)
    dh1 = da2 @ W2r.T
    da1 = dh1 * (a1 > 0)
    gW1 = F.T @ da1
    gb1 = da1.sum(0)
    return np.concatenate([g.ravel() for g in (gW1, gb1, gW2, gb2, gW3, gb3)])


def pinball(pred: np.ndarray, target: np.ndarray, levels=LEVELS):
    """Mean over pairs and levels of rho_tau(target - pred), and d/dpred."""
    u = target - pred
    tau = np.asarray(levels)[None, :]
    loss = np.where(u >= 0, tau * u, (tau - 1.0) * u)
    P, Q = pred.shape
    dpred = -np.where(u >= 0, tau, tau - 1.0) / (P * Q)
    return loss.mean(), dpred


def adam(params, grad, m, v, t, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
    m = b1 * m + (1 - b1) * grad
    v = b2 * v + (1 - b2) * grad * grad
    mh = m / (1 - b1 ** t)
    vh = v / (1 - b2 ** t)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v


def null_quantiles(T: np.ndarray, levels=LEVELS) -> np.ndarray:
    """Empirical quantiles of |T_b|: the ceil(level * B)-th smallest value."""
    a = np.sort(np.abs(np.asarray(T, dtype=np.float64)))
    B = len(a)
    return np.array([a[max(0, math.ceil(lv * B) - 1)] for lv in levels])


def predict_p(q: np.ndarray, T_obs_abs: float, levels=LEVELS) -> float:
    """p from predicted quantiles (made non-decreasing): 1 - F(|T_obs|) with F
    linear between (q_k, level_k); below q_1 linear from (0, 0); above q_9
    the last segment's slope continued, floored at 1e-4."""
    q = np.maximum.accumulate(np.asarray(q, dtype=np.float64))
    t = float(T_obs_abs)
    lv = np.asarray(levels, dtype=np.float64)
    if t <= q[0]:
        F = lv[0] * (t / q[0] if q[0] > 0 else 1.0)
    elif t >= q[-1]:
        span = max(q[-1] - q[-2], 1e-12)
        F = lv[-1] + (1 - lv[-1]) * min(1.0, (t - q[-1]) / span)
        F = min(F, 1.0 - 1e-4)
    else:
        k = int(np.searchsorted(q, t, side="right")) - 1
        k = min(max(k, 0), len(q) - 2)
        w = (t - q[k]) / max(q[k + 1] - q[k], 1e-12)
        F = lv[k] + w * (lv[k + 1] - lv[k])
    return 1.0 - F
