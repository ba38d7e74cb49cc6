"""Design-level sanity checks of the fixed-space test on synthetic clouds
(Sec. 3.1 and the split-half diagnostic of the appendix: under H0 -- equal
dispersion, mean directions free -- the aligned test is to keep its Type-I
rate):

- split-half: both groups drawn around the same direction with the same
  dispersion; p must look uniform and the aligned and naive tests must agree
  (the reflection is then close to the identity);
- the aligned test keeps its rejection rate at alpha when the two mean
  directions differ (the paper claims control of the Type-I rate, not
  uniformity of p: after the reflection the two sample mean directions
  coincide exactly, so the pooled rows are only approximately exchangeable,
  and p is measurably non-uniform at 60 degrees while the rate at alpha holds).

Each check runs 300 pairs (n = m = 200, d = 768 BF16, B = 999) through the
batched GPU path; thresholds allow about 2.5 binomial standard deviations."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2605_08048_gb300 import hbperm as H  # noqa: E402
from paper_2605_08048_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu

PAIRS, N_G, D, B, ALPHA = 300, 200, 768, 999, 0.05


@pytest.fixture(scope="module")
def ctx():
    c = H.Context(0)
    yield c
    c.close()


def batch_at(angle, seed):
    parts = []
    for k in range(PAIRS):
        X, Y = synth.pair(seed, N_G, N_G, D, 0.35, 0.35, angle, "bf16", key=k)
        parts += [X, Y]
    XY = np.concatenate(parts)
    t = torch.from_numpy(XY.view(np.int16)).view(torch.bfloat16).cuda()
    n = np.full(PAIRS, N_G, dtype=np.int64)
    return t, n, n.copy()


def pvals(ctx, XY, n, m, align):
    res = H.hb_perm_test_batched(ctx, XY, n, m, H.make_opts(B=B, seed=11, align=align))
    return np.array([r["p"] for r in res])


def ks_uniform(p):
    """Kolmogorov-Smirnov distance to U(0, 1) and its asymptotic p-value."""
    x = np.sort(p)
    k = len(x)
    dist = max(np.max(np.arange(1, k + 1) / k - x), np.max(x - np.arange(k) / k))
    lam = (np.sqrt(k) + 0.12 + 0.11 / np.sqrt(k)) * dist
    j = np.arange(1, 101)
    return dist, float(np.clip(2 * np.sum((-1) ** (j - 1) * np.exp(-2 * j * j * lam * lam)), 0, 1))


def test_split_half_null_is_uniform_and_aligned_matches_naive(ctx):
    XY, n, m = batch_at(0.0, 2001)
    pa = pvals(ctx, XY, n, m, 1)
    pn = pvals(ctx, XY, n, m, 0)
    dist, ks_p = ks_uniform(pa)
    rate = float(np.mean(pa <= ALPHA))
    print(f"\nsplit-half: aligned rejection {rate:.3f}, KS {dist:.3f} (p {ks_p:.3f}); "
          f"naive rejection {np.mean(pn <= ALPHA):.3f}; mean |p_aligned - p_naive| {np.mean(np.abs(pa - pn)):.4f}, "
          f"corr {np.corrcoef(pa, pn)[0, 1]:.4f}")
    assert ks_p > 1e-3
    assert 0.015 <= rate <= 0.095
    assert np.mean(np.abs(pa - pn)) < 0.05 and np.corrcoef(pa, pn)[0, 1] > 0.9


def test_aligned_test_keeps_its_rate_across_directions(ctx):
    XY, n, m = batch_at(60.0, 2002)
    pa = pvals(ctx, XY, n, m, 1)
    pn = pvals(ctx, XY, n, m, 0)
    dist, ks_p = ks_uniform(pa)
    rate = float(np.mean(pa <= ALPHA))
    dn, ks_n = ks_uniform(pn)
    print(f"\n60 degrees: aligned rejection {rate:.3f}, KS {dist:.3f} (p {ks_p:.2e}); "
          f"naive rejection {np.mean(pn <= ALPHA):.3f}, KS {dn:.3f} (p {ks_n:.2e})")
    assert 0.015 <= rate <= 0.095
    assert np.mean(pa <= 0.01) <= 0.035  # no excess at the paper's alpha = 0.01 either
