"""hb_align_noalloc: the allocation-free alignment entry point.

It exists for callers that cannot call cudaMalloc (device memory fully held by
their own pool allocator, or code that cannot take cudaMalloc's implicit
synchronisation); it takes its scratch from a fixed device array instead of a
context workspace.  Through the C ABI, two calls in a row -- the second on a
different, differently shaped pair, so stale contents of the shared scratch
would show -- must give exactly what hb_align gives and exactly the FP64
oracle's aligned Z and axis u.  This file is collected last and also passes
alone in a fresh process (the first call then performs the one-time address
look-up of the scratch array)."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import oracle as O  # noqa: E402
from paper_2605_08048_gb300 import hbperm as H  # noqa: E402
from paper_2605_08048_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu


def _dev(a):
    if a.dtype == np.uint16:
        return torch.from_numpy(np.ascontiguousarray(a).view(np.int16)).view(torch.bfloat16).cuda()
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _bits(t):
    return t.view(torch.int16).cpu().numpy() if t.dtype == torch.bfloat16 else t.view(torch.int32).cpu().numpy()


def _obits(a):
    return a.view(np.int16) if a.dtype == np.uint16 else a.view(np.int32)


def test_noalloc_align_equals_hb_align_and_oracle_on_two_calls_in_a_row():
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
        st, Zo, uo, _, sko = O.align(X, Y, align=align, reflect_side=side)
        assert st == 0 and skn == skr == sko == 0
        assert (_bits(Zn) == _obits(Zo)).all()  # bit-exact against the FP64 oracle
        assert (_bits(Zn) == _bits(Zr)).all()
        assert np.array_equal(un.cpu().numpy().view(np.int64), uo.view(np.int64))
        assert torch.equal(un, ur)
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch_and_null_pointers():
    X, Y = synth.pair(903, 20, 20, 2048, 0.35, 0.35, None, "bf16")
    with pytest.raises(H.HbError) as e:
        H.hb_align_noalloc(_dev(X), _dev(Y))
    assert e.value.status == H.HB_ERR_UNSUPPORTED
    assert "1024" in str(e.value)
    # a NULL output pointer through the raw C ABI: an argument error with its own message
    L = H.lib()
    X, Y = synth.pair(904, 8, 8, 64, 0.35, 0.35, None, "bf16")
    Xd, Yd = _dev(X), _dev(Y)
    st = L.hb_align_noalloc(Xd.data_ptr(), 8, Yd.data_ptr(), 8, 64, H.HB_BF16, 1, 0, None, None, None, None)
    assert st == H.HB_ERR_INVALID_ARG
    msg = L.hb_last_error().decode()
    assert "hb_align_noalloc" in msg and "NULL" in msg
