"""hb_align_noalloc: the allocation-free alignment entry point.

It exists for callers that cannot call cudaMalloc (device memory fully held by
their own pool allocator, or code that cannot take cudaMalloc's implicit
synchronisation); it takes its scratch from a fixed device array instead of a
context workspace.  Through the C ABI, two calls in a row -- the second on a
different, differently shaped pair, so stale contents of the shared scratch
would show -- must give exactly what hb_align gives.  This file is collected
last and also passes alone in a fresh process (the first call then performs
the one-time address look-up of the scratch array)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2605_08048_gb300 import hbperm as H  # noqa: E402
from paper_2605_08048_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


def _dev(a):
    if a.dtype == np.uint16:
        return torch.from_numpy(np.ascontiguousarray(a).view(np.int16)).view(torch.bfloat16).cuda()
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _bits(t):
    return t.view(torch.int16).cpu().numpy() if t.dtype == torch.bfloat16 else t.view(torch.int32).cpu().numpy()


def test_noalloc_align_equals_hb_align_on_two_calls_in_a_row():
    ctx = H.Context(0)
    cases = [
        (synth.pair(901, 300, 350, 768, 0.35, 0.40, None, "bf16"), 1, 0),
        (synth.pair(902, 57, 130, 200, 0.35, 0.35, 70.0, "f32"), 1, 1),
    ]
    for (X, Y), align, side in cases:
        Xd, Yd = _dev(X), _dev(Y)
        Zr, ur, skr = H.hb_align(ctx, Xd, Yd, align=align, reflect_side=side)
        Zn, un, skn = H.hb_align_noalloc(Xd, Yd, align=align, reflect_side=side)
        torch.cuda.synchronize()
        assert skn == skr == 0
        assert (_bits(Zn) == _bits(Zr)).all()  # the alignment is bit-exact in both entry points
        assert torch.equal(un, ur)
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    X, Y = synth.pair(903, 20, 20, 2048, 0.35, 0.35, None, "bf16")
    with pytest.raises(H.HbError) as e:
        H.hb_align_noalloc(_dev(X), _dev(Y))
    assert e.value.status == H.HB_ERR_UNSUPPORTED
    assert "1024" in str(e.value)
