"""Batched exact counting of many uneven graphs (one bfc_exact_batch call).

    python -m paper_1801_00338_gb300.batch_eval [--small]

Default workload: 4,096 Chung-Lu graphs with m log-uniform in [10^3, 10^6],
|V|/|U| uniform in [0.2, 5], exponent uniform in [1.9, 3.0] on both sides,
mean degree 8 (seed 5).  One call counts every graph: host edge lists in,
per-graph B and start side out.  The timed region is the whole call (the
host-to-device copy of the edge lists included).  Prints one JSON object:
graphs/s, edges/s and wedges/s (W of every graph at its own Algorithm 1
start side), and a check of the smallest graphs against the exact counts of
independent per-graph calls.
"""
from __future__ import annotations

import json
import sys
import time

import numpy as np

from . import bfc, synth


def wedges_at_start_side(u, v, nU, nV) -> int:
    """W of one graph: wedges centred on the side that does not start (Lemma 2),
    the start side chosen as Algorithm 1 does."""
    dU = np.bincount(u, minlength=nU).astype(np.float64)
    dV = np.bincount(v, minlength=nV).astype(np.float64)
    mid = dU if (dU * dU).sum() < (dV * dV).sum() else dV
    return int((mid * (mid - 1) / 2).sum())


def _make(args):
    i, nU, nV, m, gamma = args
    u, v = synth.chung_lu_bipartite(nU, nV, m, gamma, gamma, 100_000 + i)
    return u, v, nU, nV, wedges_at_start_side(u, v, nU, nV)


def _one_thread():
    import torch
    torch.set_num_threads(1)


def generate(count: int, seed: int, m_lo: float, m_hi: float, workers: int = 0):
    """The batch's graphs and W of each, generated by a pool of worker
    processes (spawned, so that no worker inherits a CUDA context)."""
    import multiprocessing as mp
    import os
    params = synth.uneven_batch_params(count, seed, m_lo, m_hi)
    jobs = [(i, nU, nV, m, gamma) for i, (nU, nV, m, gamma) in enumerate(params)]
    workers = workers or min(16, os.cpu_count() or 1)
    if workers > 1:
        with mp.get_context("spawn").Pool(workers, initializer=_one_thread) as pool:
            out = pool.map(_make, jobs, chunksize=8)
    else:
        out = [_make(j) for j in jobs]
    graphs = [o[:4] for o in out]
    return graphs, int(sum(o[4] for o in out))


def run(count: int, seed: int, m_lo: float, m_hi: float, reps: int = 3) -> dict:
    t0 = time.perf_counter()
    graphs, W = generate(count, seed, m_lo, m_hi)
    gen_s = time.perf_counter() - t0
    import torch
    edges = int(sum(len(g[0]) for g in graphs))
    bfc.bfc_exact_batch(graphs)  # warm-up (allocator pool, library load)
    times = []
    for _ in range(reps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        B, side = bfc.bfc_exact_batch(graphs)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    dt = float(np.median(times))
    # the smallest graphs, one call each, must give the same counts
    small = np.argsort([len(g[0]) for g in graphs])[:32]
    ok = True
    for i in small:
        u, v, nU, nV = graphs[i]
        with bfc.Graph(u, v, nU, nV) as G:
            ok &= G.exact()[0] == int(B[i])
    return {"graphs": count, "m_range": [m_lo, m_hi], "edges": edges, "W": int(W), "gen_s": gen_s,
            "s_per_call": dt, "s_all": times, "graphs_per_s": count / dt, "edges_per_s": edges / dt,
            "wedges_per_s": W / dt, "B_total": int(B.astype(np.float64).sum()),
            "smallest_32_equal_single_calls": bool(ok)}


if __name__ == "__main__":
    if "--small" in sys.argv:
        print(json.dumps(run(256, 5, 1e3, 1e5)))
    else:
        print(json.dumps(run(4096, 5, 1e3, 1e6)))
