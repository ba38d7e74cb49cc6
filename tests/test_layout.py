"""Host-side launch layout of a batched call (hb_plan_layout; no GPU): row
chunks, input pieces, the GEMM work list and the label/GEMM chunk cuts hold
the invariants the kernels rely on."""
import os
import shutil

import numpy as np
import pytest

from paper_2605_08048_gb300 import hbperm as H

CHUNK_ROWS, PIECES, S1_MAX = 128, 8, 65536
# relabellings per work item: one 128-row tile for single CTAs, two for CTA pairs
CLUSTER_TILES = {H.HB_PATH_MIXED: 128, H.HB_PATH_MIXED_NARROW: 128, H.HB_PATH_MIXED_2SM: 2 * 128}


@pytest.fixture(scope="module", autouse=True)
def built():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("no CUDA toolkit")
    from paper_2605_08048_gb300 import build
    return build.build()


def lognormal_sizes(seed, P):
    rng = np.random.default_rng(seed)
    s = np.clip(np.round(np.exp(rng.normal(np.log(300), 1.0, (2, P)))), 20, 8000).astype(np.int64)
    return s[0], s[1]


CASES = {
    "tiny": ([2, 3], [2, 5]),
    "ragged": ([5, 300, 40, 1, 129, 128, 127, 4], [7, 129, 1000, 9, 3, 128, 2, 2]),
    "one_big": ([4000] + [30] * 20, [3000] + [25] * 20),
    "lognormal": lognormal_sizes(5, 300),
    "no_work": ([1, 5, 1], [9, 1, 1]),  # every pair has n < 2 or m < 2: no work items
    "both_modes": ([5000, 30, 8000, 4096], [4000, 40, 200, 4096]),  # n + m above and at the single-slice limit
}


def rup(x, k):
    return (x + k - 1) // k * k


@pytest.mark.parametrize("case", list(CASES))
@pytest.mark.parametrize("path", [H.HB_PATH_MIXED, H.HB_PATH_MIXED_NARROW, H.HB_PATH_MIXED_2SM, H.HB_PATH_FP32_PLAIN])
@pytest.mark.parametrize("dtype", [H.HB_BF16, H.HB_F32])
def test_layout_invariants(case, path, dtype):
    n, m = (np.asarray(v, dtype=np.int64) for v in CASES[case])
    P, B = len(n), 999
    lay = H.plan_layout(n, m, 768, dtype, H.make_opts(B=B, path=path))
    ch, pc = lay["chunks"], lay["pieces"]

    # row chunks: pair-major, X rows then Y rows, each side covered in order by
    # chunks of at most CHUNK_ROWS rows; every chunk starts at a token index t
    # with (t mod 32) + rows <= CHUNK_ROWS (a warp covers four 32-token groups)
    first = np.zeros(P + 1, dtype=np.int64)
    k = 0
    for p in range(P):
        first[p] = k
        for side, rows in ((0, n[p]), (1, m[p])):
            r0 = 0
            while r0 < rows:
                pair, sd, row0, nr = ch[k]
                assert (pair, sd, row0) == (p, side, r0) and 1 <= nr <= CHUNK_ROWS
                tok0 = (n[p] if side else 0) + row0
                assert tok0 % 32 + nr <= CHUNK_ROWS
                r0 += nr
                k += 1
            assert r0 == rows
    first[P] = k
    assert k == len(ch)

    # input pieces: at most PIECES, non-empty, a contiguous cover of the pairs
    # and of their chunks, cut near equal shares of the rows
    assert 1 <= len(pc) <= min(PIECES, P)
    assert pc[0][0] == 0 and pc[-1][1] == P
    N = n + m
    for a, b in zip(pc[:-1], pc[1:]):
        assert a[1] == b[0]
    for p0, p1, c0, c1 in pc:
        assert p0 < p1 and c0 == first[p0] and c1 == first[p1]
        assert N[p0:p1].sum() <= N.sum() / PIECES + N.max() + 1

    if path == H.HB_PATH_FP32_PLAIN:
        assert len(lay["items"]) == 0 and len(lay["label_chunks"]) == 1 and len(lay["order"]) == 0
        return
    # work list: pairs by padded size, largest first (ties in pair order), each
    # valid pair's relabelling groups in order
    order, items, lc = lay["order"], lay["items"], lay["label_chunks"]
    assert sorted(order) == list(range(P))
    key = [(-rup(N[p], 64), p) for p in order]
    assert key == sorted(key)
    tiles = CLUSTER_TILES[path]
    groups = rup(B, tiles) // tiles
    valid = [p for p in order if n[p] >= 2 and m[p] >= 2]
    # BF16 pairs up to the single-slice limit run the single-slice pass (mode 1)
    mode = {p: int(dtype == H.HB_BF16 and N[p] <= S1_MAX) for p in valid}
    want = [(p, g, mode[p]) for p in valid for g in range(groups)]
    assert [tuple(x) for x in items] == want
    if not valid:
        assert len(items) == 0 and len(order) == P  # the order is written even with no work items
        return
    # label / GEMM chunks: cuts along `order`, the items of each chunk's pairs,
    # the first chunk the shortest prefix holding 16 % of the label words
    pos, it = lc[:, 0], lc[:, 1]
    assert pos[0] == 0 and pos[-1] == P and (np.diff(pos) > 0).all() and len(lc) <= 5
    for c in range(len(lc) - 1):
        seg = [p for p in order[pos[c]:pos[c + 1]] if n[p] >= 2 and m[p] >= 2]
        assert it[c + 1] - it[c] == groups * len(seg)
    words = np.array([((N[p] + 31) // 32) * rup(B, tiles) for p in order])
    if len(lc) > 2:
        assert words[:pos[1]].sum() >= words.sum() * 16 // 100 > words[:pos[1] - 1].sum()


def test_layout_argument_checks():
    o = H.make_opts(B=99)
    with pytest.raises(H.HbError) as e:
        H.plan_layout([10], [10], 64, H.HB_BF16, H.make_opts(B=99, path=H.HB_PATH_AUTO))
    assert e.value.status == H.HB_ERR_INVALID_ARG
    with pytest.raises(H.HbError) as e:
        H.plan_layout([0, 5], [5, 5], 64, H.HB_BF16, o)
    assert e.value.status == H.HB_ERR_INVALID_ARG
    with pytest.raises(H.HbError) as e:
        H.plan_layout([40000], [30000], 64, H.HB_BF16, o)
    assert e.value.status == H.HB_ERR_UNSUPPORTED
    with pytest.raises(H.HbError) as e:
        H.plan_layout([10], [10], 0, H.HB_BF16, o)
    assert e.value.status == H.HB_ERR_INVALID_ARG
