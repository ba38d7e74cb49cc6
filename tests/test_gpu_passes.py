"""The tensor-core passes and the bounded device waits.

BF16 pairs up to the single-slice limit are decided by the first grid slice
alone where that pass's error band allows, then by both slices for the
relabellings it lists, then exactly; larger pairs take both slices at once.
Counts and p must equal the oracle's whichever pass decides (Algorithm 1,
Eq. pvalue), on every route, with the single-slice pass forced onto pairs
whose band is wide (many relabellings gathered) and switched off.

Every mbarrier wait of the tensor-core kernels is bounded: with one arrival
withheld (a test hook; nothing then completes that barrier) the wait runs
out, the call returns HB_ERR_TIMEOUT, and the next call on the same context
gives the oracle's results again.

Every case also runs on CTA pairs with the label operand in tensor memory
(HB_OPT_A_OPERAND_TMEM: tcgen05.st by the producer warps, 192-column
accumulator tiles)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2605_08048_gb300 import hbperm as H  # noqa: E402
from paper_2605_08048_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu

ROUTES = [pytest.param((H.HB_PATH_MIXED, 0), id="mixed"), pytest.param((H.HB_PATH_MIXED_2SM, 0), id="mixed-2sm"),
          pytest.param((H.HB_PATH_MIXED_2SM, 1), id="mixed-2sm-tmem"),
          pytest.param((H.HB_PATH_MIXED_NARROW, 0), id="mixed-narrow")]


def dev(a: np.ndarray):
    if a.dtype == np.uint16:
        return torch.from_numpy(np.ascontiguousarray(a).view(np.int16)).view(torch.bfloat16).cuda()
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def ctx():
    c = H.Context(0)
    yield c
    c.close()


def _set(ctx, s1_max=65536, wait_ns=4_000_000_000, a_tmem=0):
    H.set_option(ctx, H.HB_OPT_SINGLE_SLICE_MAX_N, s1_max)
    H.set_option(ctx, H.HB_OPT_WAIT_LIMIT_NS, wait_ns)
    H.set_option(ctx, H.HB_OPT_A_OPERAND_TMEM, a_tmem)


@pytest.mark.parametrize("route", ROUTES)
@pytest.mark.parametrize("s1_max", [0, 65536], ids=["two-slice-only", "single-slice-first"])
def test_passes_parity_wide_band(ctx, route, s1_max):
    """A null pair of 6000 tokens: its single-slice band is wide, so the
    gathered pass decides many relabellings; counts, p and the statistics of
    every relabelling agree with the oracle."""
    path, tm = route
    _set(ctx, s1_max=s1_max, a_tmem=tm)
    X, Y = synth.pair(4321, 3100, 2900, 768, 0.35, 0.35, None, "bf16")
    B = 1500
    ref, Tref, _ = O.perm_test(X, Y, O.opts(B=B, seed=9), want_T=True)
    res, T = H.hb_perm_test(ctx, dev(X), dev(Y), H.make_opts(B=B, seed=9, path=path), want_T=True)
    _set(ctx)
    assert res["status"] == 0
    assert res["count"] == ref["count"] and res["p"] == ref["p"]
    assert np.abs(T.cpu().numpy().astype(np.float64) - Tref).max() <= 2e-4
    assert res["n_rechecked"] <= 0.01 * B


@pytest.mark.parametrize("route", ROUTES)
def test_passes_parity_batch_mixed_sizes(ctx, route):
    """Pairs on both sides of the single-slice limit in one batch (limit set
    to 600 tokens), ragged sizes, one degenerate pair."""
    path, tm = route
    _set(ctx, s1_max=600, a_tmem=tm)
    n = np.array([300, 2, 1, 700, 45, 1000, 260], dtype=np.int64)
    m = np.array([250, 9, 30, 20, 3000, 990, 340], dtype=np.int64)
    b = synth.batch(77, len(n), 256, "bf16", sizes=(n, m))
    res = H.hb_perm_test_batched(ctx, dev(b.XY), n, m, H.make_opts(B=999, seed=4, path=path), check=False)
    _set(ctx)
    ref = O.perm_test_batched(b.XY, n, m, O.opts(B=999, seed=4))
    for r, q in zip(res, ref):
        assert r["status"] == q["status"]
        if q["status"] == 0:
            assert r["count"] == q["count"] and r["p"] == q["p"]


@pytest.mark.parametrize("route", ROUTES)
def test_bounded_wait_timeout_then_recovery(ctx, route):
    path, tm = route
    X, Y = synth.pair(555, 700, 900, 768, 0.35, 0.385, None, "bf16")
    Xd, Yd = dev(X), dev(Y)
    opts = H.make_opts(B=3000, seed=12, path=path)
    _set(ctx, wait_ns=50_000_000, a_tmem=tm)
    H.set_option(ctx, H.HB_OPT_TEST_WITHHOLD_ARRIVAL, 1)
    with pytest.raises(H.HbError) as e:
        H.hb_perm_test(ctx, Xd, Yd, opts)
    assert e.value.status == H.HB_ERR_TIMEOUT
    # the hook acts on one call; the same context then gives the oracle's results
    _set(ctx, a_tmem=tm)
    res, _ = H.hb_perm_test(ctx, Xd, Yd, opts)
    ref, _, _ = O.perm_test(X, Y, O.opts(B=3000, seed=12))
    assert res["status"] == 0 and res["count"] == ref["count"] and res["p"] == ref["p"]
    _set(ctx)


def test_option_checks(ctx):
    with pytest.raises(H.HbError) as e:
        H.set_option(ctx, H.HB_OPT_WAIT_LIMIT_NS, 10)
    assert e.value.status == H.HB_ERR_INVALID_ARG
    with pytest.raises(H.HbError) as e:
        H.set_option(ctx, 99, 1)
    assert e.value.status == H.HB_ERR_INVALID_ARG
