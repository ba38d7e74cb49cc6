"""Writes the oracle's results for every pair of the batched benchmark workload.

The workload is the one the benchmark times: 4096 pairs with lognormal sizes
(median 300, sigma_log 1.0, clipped 20..8000), d = 768 BF16, half null and half
alternative (synth.workload_batched, data seed 1237), B = 9999 relabellings
with Philox seed 1, Householder-aligned, two-sided log-volume statistic.  Each
line of the output holds one pair: index, n, m, status, count, p (repr of the
double).  Only the FP64/exact CPU oracle computes these values (Algorithm 1;
Eq. pvalue); the GPU test compares every pair's count and p with them.

Run from the repository root:  python tests/golden/make_batched4096_oracle.py
It resumes an interrupted run from the lines already written.
"""
from __future__ import annotations

import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

from oracle import oracle as O  # noqa: E402
from paper_2605_08048_gb300 import synth  # noqa: E402

OUT = os.path.join(HERE, "batched4096_b9999_oracle.txt")
P, B, SEED, DATA_SEED = 4096, 9999, 1, 1237
HEADER = (f"# oracle results, batched workload: P={P}, data seed {DATA_SEED} (synth.workload_batched), d=768 BF16, "
          f"B={B}, Philox seed {SEED}, align=1, two-sided log-volume\n# pair n m status count p\n")


def main():
    done = 0
    if os.path.exists(OUT):
        done = sum(1 for line in open(OUT) if line and not line.startswith("#"))
    else:
        with open(OUT, "w") as f:
            f.write(HEADER)
    if done >= P:
        print("complete")
        return
    batch = synth.workload_batched(seed=DATA_SEED, P=P)
    off = batch.offsets
    o = O.opts(B=B, seed=SEED)
    t0 = time.time()
    step = 32
    for p0 in range(done, P, step):
        p1 = min(P, p0 + step)
        XY = np.ascontiguousarray(batch.XY[off[p0]:off[p1]])
        res = O.perm_test_batched(XY, batch.n[p0:p1], batch.m[p0:p1], o)
        with open(OUT, "a") as f:
            for k, r in enumerate(res):
                p = p0 + k
                f.write(f"{p} {batch.n[p]} {batch.m[p]} {r['status']} {r['count']} {r['p']!r}\n")
        print(f"{p1}/{P} pairs, {time.time() - t0:.0f} s", flush=True)


if __name__ == "__main__":
    main()
