"""GPU tests of the routes and the route tuner: the narrow tensor-core
route, the SIMT route for pairs above the tensor-core size limit, and
HB_PATH_AUTO splitting one batch over routes, all with results identical to
a single forced route (and so to the oracle, which the parity tests tie
every route to)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2605_08048_gb300 import hbperm as H  # noqa: E402
from paper_2605_08048_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu

KEYS = ("p", "count", "B_eff", "T_obs", "r_x", "r_y", "reflection_skipped", "status", "n_rechecked")


def dev(a: np.ndarray):
    if a.dtype == np.uint16:
        return torch.from_numpy(np.ascontiguousarray(a).view(np.int16)).view(torch.bfloat16).cuda()
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture()
def ctx():
    c = H.Context(0)  # a fresh route table per test
    yield c
    c.close()


def same_decision(a, b):
    return all(x[k] == y[k] for x, y in zip(a, b) for k in ("p", "count", "B_eff", "T_obs", "status"))


def test_untuned_routes(ctx):
    assert H.route(ctx, 2) == H.HB_PATH_MIXED_2SM
    assert H.route(ctx, 65536) == H.HB_PATH_MIXED_2SM
    assert H.route(ctx, 65537) == H.HB_PATH_FP32_PLAIN
    assert H.route(ctx, 1 << 20) == H.HB_PATH_FP32_PLAIN
    with pytest.raises(H.HbError):
        H.route(ctx, 1)
    with pytest.raises(H.HbError):
        H.route(ctx, (1 << 20) + 1)


def test_auto_sends_large_pairs_to_simt(ctx):
    # one pair above the tensor-core limit of n + m = 65536, three below
    sizes = ([120, 35000, 30, 500], [90, 35001, 64, 700])
    b = synth.batch(101, 4, d=64, dtype="bf16", sizes=sizes)
    XY = dev(b.XY)
    with pytest.raises(H.HbError) as e:
        H.hb_perm_test_batched(ctx, XY, b.n, b.m, H.make_opts(B=199, seed=2, path=H.HB_PATH_MIXED))
    assert e.value.status == H.HB_ERR_UNSUPPORTED
    auto = H.hb_perm_test_batched(ctx, XY, b.n, b.m, H.make_opts(B=199, seed=2, path=H.HB_PATH_AUTO))
    plain = H.hb_perm_test_batched(ctx, XY, b.n, b.m, H.make_opts(B=199, seed=2, path=H.HB_PATH_FP32_PLAIN))
    assert same_decision(auto, plain)
    # the small pairs alone on the tensor cores agree as well
    small = [0, 2, 3]
    bs = synth.Batch(np.concatenate([b.XY[b.offsets[p]:b.offsets[p + 1]] for p in small]), b.n[small], b.m[small],
                     b.d, b.dtype, b.null[small])
    mixed = H.hb_perm_test_batched(ctx, dev(bs.XY), bs.n, bs.m, H.make_opts(B=199, seed=2, path=H.HB_PATH_MIXED))
    assert same_decision([auto[p] for p in small], mixed)
    # host input through the route split
    auto_h = H.hb_perm_test_batched(ctx, XY.cpu(), b.n, b.m, H.make_opts(B=199, seed=2, path=H.HB_PATH_AUTO))
    assert same_decision(auto_h, auto)
    X, Y = b.pair(2)
    r, _, _ = O.perm_test(X, Y, O.opts(B=199, seed=2))
    assert auto[2]["count"] == r["count"]


def test_autotune_fills_the_route_table(ctx):
    opts = H.make_opts(B=255, seed=1)
    ms = H.autotune(ctx, 128, torch.bfloat16, opts, max_N=1024)
    assert ms.shape == (H.ROUTE_BUCKETS, len(H.ROUTE_PATHS))
    assert (ms[:5] > 0).all() and (ms[5:] == -1).all()  # buckets up to N = 1024 timed
    for k in range(5):
        N = 64 << k
        assert H.route(ctx, N) == H.ROUTE_PATHS[int(np.argmin(ms[k]))]
    assert H.route(ctx, 70000) == H.HB_PATH_FP32_PLAIN
    b = synth.batch(102, 6, d=128, dtype="bf16", sizes=([20, 60, 200, 400, 33, 700], [30, 64, 180, 500, 31, 300]))
    XY = dev(b.XY)
    auto = H.hb_perm_test_batched(ctx, XY, b.n, b.m, H.make_opts(B=999, seed=4, path=H.HB_PATH_AUTO))
    ref = H.hb_perm_test_batched(ctx, XY, b.n, b.m, H.make_opts(B=999, seed=4, path=H.HB_PATH_MIXED))
    assert same_decision(auto, ref)
    plan = H.Plan(ctx, b.n, b.m, 128, torch.bfloat16, H.make_opts(B=999, seed=4, path=H.HB_PATH_AUTO))
    assert same_decision(plan.execute(XY), ref)
    plan.close()


def test_single_pair_auto(ctx):
    b = synth.batch(103, 1, d=96, dtype="f32", sizes=([150], [170]))
    X, Y = b.pair(0)
    Xd, Yd = dev(X), dev(Y)
    r1, _ = H.hb_perm_test(ctx, Xd, Yd, H.make_opts(B=999, seed=9, path=H.HB_PATH_AUTO))
    r2, _ = H.hb_perm_test(ctx, Xd, Yd, H.make_opts(B=999, seed=9, path=H.HB_PATH_FP32_PLAIN))
    assert r1["count"] == r2["count"] and r1["p"] == r2["p"]
