"""The multi-GPU host logic on CPU: two gloo ranks shard a batch of pairs,
test their shares (here with the CPU oracle standing in for the GPU path)
and gather every result in pair order; the result equals one process testing
the whole batch.  Also the sharding's balance and coverage, and the
max-over-ranks timing."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from oracle import oracle as O  # noqa: E402
from paper_2605_08048_gb300 import shard as S  # noqa: E402
from paper_2605_08048_gb300 import synth  # noqa: E402

SIZES = ([20, 7, 30, 3, 12, 40, 5, 9], [15, 25, 6, 4, 12, 33, 5, 21])
OPTS = dict(B=199, seed=4)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = synth.batch(55, len(SIZES[0]), d=32, dtype="f32", sizes=SIZES)

        def runner(XY, n, m):
            return O.perm_test_batched(XY, n, m, O.opts(**OPTS))

        res = S.run_sharded(runner, b.XY, b.n, b.m, rank, world)
        slowest = S.max_over_ranks(0.5 + rank)
        np.save(os.path.join(out_dir, f"r{rank}.npy"),
                np.array([[r["count"] for r in res], [r["p"] for r in res]] + [[slowest] * len(res)]))
    finally:
        dist.destroy_process_group()


def test_shard_balances_and_covers():
    rng = np.random.default_rng(3)
    n = rng.integers(2, 5000, 997)
    m = rng.integers(2, 5000, 997)
    for world in (1, 2, 3, 8):
        parts = S.shard(n, m, world)
        allidx = np.sort(np.concatenate(parts))
        assert np.array_equal(allidx, np.arange(997))
        loads = np.array([np.sum(n[p] + m[p]) for p in parts])
        assert loads.max() - loads.min() <= np.max(n + m)  # longest-first greedy bound
        assert all(np.all(np.diff(p) > 0) for p in parts)


def test_pack_extracts_the_pairs_rows():
    b = synth.batch(56, 5, d=8, dtype="f32", sizes=([3, 4, 5, 6, 7], [2, 3, 4, 5, 6]))
    sub, ns, ms = S.pack(b.XY, b.n, b.m, np.array([1, 3]))
    assert list(ns) == [4, 6] and list(ms) == [3, 5]
    X1, Y1 = b.pair(1)
    X3, Y3 = b.pair(3)
    assert np.array_equal(sub, np.concatenate([X1, Y1, X3, Y3]))
    st, _, _ = S.pack(torch.from_numpy(b.XY), b.n, b.m, np.array([1, 3]))
    assert np.array_equal(st.numpy(), sub)


def test_two_gloo_ranks_equal_one_process(tmp_path):
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    b = synth.batch(55, len(SIZES[0]), d=32, dtype="f32", sizes=SIZES)
    ref = O.perm_test_batched(b.XY, b.n, b.m, O.opts(**OPTS))
    for rank in range(world):
        got = np.load(tmp_path / f"r{rank}.npy")
        assert list(got[0].astype(np.int64)) == [r["count"] for r in ref]
        assert list(got[1]) == [r["p"] for r in ref]
        assert np.all(got[2] == 1.5)  # the slowest rank's time on every rank

