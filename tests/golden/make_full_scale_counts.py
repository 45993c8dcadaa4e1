"""Write the oracle's exact counts of two large seeded workloads (test data).

    python tests/golden/make_full_scale_counts.py [--procs N] [--only sparsify|batch]

Only oracle/ computes here (the CUDA library is not used), on the host's
cores.  Inputs come from the seeded generators in the package's synth module.

  chung_lu_20m_40m_300m.txt  Chung-Lu bipartite |U| = 20M, |V| = 40M, 300M
      distinct edges, exponents 2.0 / 2.3, seed 3 (the sparsification
      estimators' workload): B by Algorithm 1's start-side choice, as
      (sum over the start side of b_v) / 2 (Eq. (1): every butterfly has two
      start-side vertices), b_v by Algorithm 2; the start vertices are split
      over forked processes that share the prepared graph.
  uneven_batch_4096.txt  4,096 Chung-Lu graphs of uneven size (the batched
      exact-count workload, synth.uneven_batch_params(4096, 5)): B and the
      start side of every graph by Algorithm 1.
"""
from __future__ import annotations

import argparse
import multiprocessing as mp
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
from paper_1801_00338_gb300 import synth  # noqa: E402

_P = None  # the prepared graph, shared with forked workers


def _part(ids):
    s, w = _P.count(ids)
    return s, w


def sparsify_workload(procs: int) -> str:
    global _P
    t0 = time.time()
    g = synth.chung_lu_scaled(20_000_000, 40_000_000, 300_000_000, 2.0, 2.3, 3)
    sqU, sqV = oracle.degree_square_sums(g.u, g.v, g.nU, g.nV)
    side = 1 if sqU < sqV else 0  # Algorithm 1: start from R when sum_L d^2 < sum_R d^2
    n = g.nV if side else g.nU
    _P = oracle.Prepared(g.u, g.v, g.nU, g.nV, side)
    m = g.m
    del g
    print(f"generated and prepared in {time.time() - t0:.0f} s; start side {'UV'[side]}", flush=True)
    chunks = [np.arange(i, n, 64 * procs, dtype=np.uint32) for i in range(64 * procs)]
    with mp.get_context("fork").Pool(procs) as pool:
        parts = pool.map(_part, chunks, chunksize=1)
    total = sum(int(s) for s, _ in parts)
    paths = sum(int(w) for _, w in parts)
    assert total % 2 == 0
    _P.close()
    print(f"counted in {time.time() - t0:.0f} s", flush=True)
    return (
        "# Chung-Lu bipartite |U|=20,000,000 |V|=40,000,000 m=300,000,000 exponents 2.0/2.3 seed 3\n"
        "# B by Algorithm 1's side choice; B = (sum over the start side of b_v) / 2 (Eq. (1)),\n"
        "# b_v by Algorithm 2 (oracle/bfc_oracle.c); written by tests/golden/make_full_scale_counts.py\n"
        f"m {m}\nstart_side {'UV'[side]}\nB {total // 2}\n2paths {paths}\n")


def _batch_one(i, params):
    u, v, nU, nV = synth.uneven_batch_graph(i, params)
    B, side = oracle.exact(u, v, nU, nV)
    return i, B, side, len(u)


def _batch_job(args):
    return _batch_one(*args)


def batch_workload(procs: int) -> str:
    t0 = time.time()
    params = synth.uneven_batch_params(4096, 5)
    res = []
    with mp.get_context("spawn").Pool(procs) as pool:
        for r in pool.imap_unordered(_batch_job, [(i, params) for i in range(len(params))], chunksize=4):
            res.append(r)
            if len(res) % 512 == 0:
                print(f"  {len(res)} graphs, {time.time() - t0:.0f} s", flush=True)
    res.sort()
    print(f"4096 graphs counted in {time.time() - t0:.0f} s", flush=True)
    lines = ["# 4,096 uneven Chung-Lu graphs: synth.uneven_batch_params(4096, 5), graph i from",
             "# synth.uneven_batch_graph(i, params); B and start side by Algorithm 1 (oracle/bfc_oracle.c);",
             "# written by tests/golden/make_full_scale_counts.py",
             "# columns: index m B start_side(0=U,1=V)"]
    lines += [f"{i} {m} {B} {side}" for i, B, side, m in res]
    return "\n".join(lines) + "\n"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--procs", type=int, default=os.cpu_count() or 1)
    ap.add_argument("--only", choices=("sparsify", "batch"))
    args = ap.parse_args()
    oracle.build()
    if args.only in (None, "batch"):
        text = batch_workload(args.procs)
        with open(os.path.join(HERE, "uneven_batch_4096.txt"), "w") as f:
            f.write(text)
    if args.only in (None, "sparsify"):
        text = sparsify_workload(args.procs)
        with open(os.path.join(HERE, "chung_lu_20m_40m_300m.txt"), "w") as f:
            f.write(text)


if __name__ == "__main__":
    main()
