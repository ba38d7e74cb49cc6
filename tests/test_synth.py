"""The synthetic-input generators (no method arithmetic): the host recipe
and its GPU twin draw the same sizes and the same cloud model."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2605_08048_gb300 import synth as SY  # noqa: E402


def test_device_batch_generator_shapes_and_norms():
    """synth.batch_device (the GPU recipe) on the CPU: sizes from the same
    lognormal recipe, unit rows within BF16 rounding, reproducible per seed."""
    b = SY.batch_device(7, 12, d=40, device="cpu")
    n, m = SY.lognormal_sizes(7, 12)
    assert list(b.n) == list(n) and list(b.m) == list(m)
    assert b.XY.shape == (int(np.sum(n + m)), 40) and b.XY.dtype == torch.bfloat16
    assert float((b.XY.float().norm(dim=1) - 1).abs().max()) < 1e-2
    assert torch.equal(SY.batch_device(7, 12, d=40, device="cpu").XY, b.XY)
    assert not torch.equal(SY.batch_device(8, 12, d=40, device="cpu").XY[:10], b.XY[:10])
    assert b.null.sum() == 6
