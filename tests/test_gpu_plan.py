"""GPU tests of planned batches (hb_plan): the captured CUDA graph of a whole
batched test gives exactly the results of the unplanned call and of the CPU
oracle, on first and repeated replays, on new inputs at other addresses and
on host inputs."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2605_08048_gb300 import hbperm as H  # noqa: E402
from paper_2605_08048_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu

PATHS = [pytest.param(H.HB_PATH_FP32_PLAIN, id="plain"), pytest.param(H.HB_PATH_MIXED, id="mixed")]
KEYS = ("p", "count", "B_eff", "T_obs", "r_x", "r_y", "reflection_skipped", "status", "n_rechecked")


def dev(a: np.ndarray):
    if a.dtype == np.uint16:
        return torch.from_numpy(np.ascontiguousarray(a).view(np.int16)).view(torch.bfloat16).cuda()
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


@pytest.fixture(scope="module")
def ctx():
    c = H.Context(0)
    yield c
    c.close()


def same(a, b):
    return all(x[k] == y[k] for x, y in zip(a, b) for k in KEYS)


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("dtype", ["bf16", "f32"])
def test_plan_equals_unplanned_call_and_oracle(ctx, path, dtype):
    b = synth.batch(71, 5, d=200, dtype=dtype, sizes=([40, 150, 3, 77, 300], [60, 90, 5, 33, 260]))
    opts = H.make_opts(B=1999, seed=7, path=path)
    XY = dev(b.XY)
    plan = H.Plan(ctx, b.n, b.m, b.d, XY.dtype, opts)
    want = H.hb_perm_test_batched(ctx, XY, b.n, b.m, opts)
    for _ in range(3):  # first and repeated replays
        got = plan.execute(XY)
        assert same(got, want)
    for p in (0, 2, 4):
        X, Y = b.pair(p)
        r, _, _ = O.perm_test(X, Y, O.opts(B=1999, seed=7))
        assert got[p]["count"] == r["count"] and got[p]["p"] == r["p"]
    plan.close()


def test_plan_rebinds_to_new_inputs_and_host_memory(ctx):
    sizes = ([120, 300, 45, 800, 64], [200, 90, 60, 700, 64])
    b1 = synth.batch(81, 5, d=768, dtype="bf16", sizes=sizes)
    b2 = synth.batch(82, 5, d=768, dtype="bf16", sizes=sizes)
    opts = H.make_opts(B=4999, seed=3)
    X1, X2 = dev(b1.XY), dev(b2.XY)
    plan = H.Plan(ctx, b1.n, b1.m, 768, torch.bfloat16, opts)
    w1 = H.hb_perm_test_batched(ctx, X1, b1.n, b1.m, opts)
    w2 = H.hb_perm_test_batched(ctx, X2, b2.n, b2.m, opts)
    assert not same(w1, w2)
    assert same(plan.execute(X1), w1)
    assert same(plan.execute(X2), w2)  # another address: pair pointers re-uploaded
    assert same(plan.execute(X1), w1)
    Xh = X2.cpu().pin_memory()
    assert same(plan.execute(Xh), w2)  # host input through the plan's device buffer
    assert same(plan.execute(X2.cpu()), w2)  # pageable host memory
    plan.close()


def test_plan_reports_stage_times(ctx):
    b = synth.batch(91, 3, d=256, dtype="bf16", sizes=([100, 200, 50], [100, 150, 70]))
    opts = H.make_opts(B=999, seed=5)
    H.set_timing(ctx, True)
    try:
        plan = H.Plan(ctx, b.n, b.m, 256, torch.bfloat16, opts)
        plan.execute(dev(b.XY))
        st, launches = H.stage_times(ctx)
        assert launches > 8
        assert all(v >= 0.0 for v in st.values()) and st["gemm_epilogue"] > 0.0
        plan.close()
    finally:
        H.set_timing(ctx, False)


def test_plan_argument_checks(ctx):
    b = synth.batch(95, 2, d=64, dtype="bf16", sizes=([10, 20], [10, 20]))
    opts = H.make_opts(B=99)
    plan = H.Plan(ctx, b.n, b.m, 64, torch.bfloat16, opts)
    with pytest.raises(ValueError):
        plan.execute(torch.zeros((60, 32), dtype=torch.bfloat16, device="cuda"))
    with pytest.raises(ValueError):
        plan.execute(torch.zeros((60, 64), dtype=torch.float32, device="cuda"))
    st = H.lib().hb_plan_execute(plan._h, None, None, None)
    assert st == H.HB_ERR_INVALID_ARG
    plan.close()
    with pytest.raises(H.HbError):
        H.Plan(ctx, [0, 5], [5, 5], 64, torch.bfloat16, opts)  # an empty group
