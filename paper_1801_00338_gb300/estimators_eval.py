"""Sparsification estimators at scale: ESpar (Algorithm 8) and ClrSpar
(Algorithm 9) trials against the exact count (Algorithm 1) of the same graph.

    python -m paper_1801_00338_gb300.estimators_eval [--small]

Default workload: Chung-Lu bipartite |U| = 20M, |V| = 40M, 300M distinct
edges, exponents 2.0 (U) / 2.3 (V), seed 3; 256 ESpar trials at p = 0.05 and
256 ClrSpar trials with 20 colours.  Prints one JSON object: the exact B and
its time, and per estimator the mean, median, relative errors, the per-trial
GPU time and the kept fraction implied by beta.
"""
from __future__ import annotations

import json
import sys
import time

import numpy as np

from . import bfc, synth


def run(nU: int, nV: int, m: int, gu: float, gv: float, seed: int, p: float, colors: int, trials: int) -> dict:
    import torch
    out = {"workload": {"nU": nU, "nV": nV, "m": m, "gamma": [gu, gv], "seed": seed},
           "espar": {"p": p, "trials": trials}, "clrspar": {"colors": colors, "trials": trials}}
    t0 = time.perf_counter()
    g = synth.chung_lu_scaled(nU, nV, m, gu, gv, seed)
    out["gen_s"] = time.perf_counter() - t0
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        G = bfc.Graph(g.u, g.v, g.nU, g.nV, stream=stream)
    del g
    try:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        B, side = G.exact(stream=stream)   # first call also builds the rank layout
        torch.cuda.synchronize()
        out["exact_first_s"] = time.perf_counter() - t0
        t0 = time.perf_counter()
        B2, _ = G.exact(stream=stream)
        torch.cuda.synchronize()
        out["exact_s"] = time.perf_counter() - t0
        assert B2 == B
        st = G.stats
        W = st["wedges_v"] if side == 0 else st["wedges_u"]
        out["exact"] = {"B": int(B), "start_side": "UV"[side], "W": int(W), "wedges_per_s": W / out["exact_s"]}
        for name, fn, arg in (("espar", G.espar, p), ("clrspar", G.clrspar, colors)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            est, beta = fn(arg, trials, 2024, stream=stream)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            est = np.asarray(est, dtype=np.float64)
            rel = np.abs(est - B) / B
            r = out[name]
            r.update({"mean": float(est.mean()), "median": float(np.median(est)),
                      "rel_err_of_mean": float(abs(est.mean() - B) / B),
                      "median_rel_err_single": float(np.median(rel)),
                      "rel_std_single": float(est.std(ddof=1) / B) if trials > 1 else None,
                      "se_of_mean_rel": float(est.std(ddof=1) / B / np.sqrt(trials)) if trials > 1 else None,
                      "total_s": dt, "s_per_trial": dt / trials,
                      "beta_mean": float(np.mean(beta.astype(np.float64)))})
    finally:
        G.close()
    return out


if __name__ == "__main__":
    if "--small" in sys.argv:
        res = run(200_000, 400_000, 3_000_000, 2.0, 2.3, 3, 0.05, 20, 64)
    else:
        res = run(20_000_000, 40_000_000, 300_000_000, 2.0, 2.3, 3, 0.05, 20, 256)
    print(json.dumps(res))
