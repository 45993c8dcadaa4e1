"""Sampling estimators at equal accuracy on one graph: the comparison of
Section 5 (time per sampling iteration, error against time; median of 30
trials as in the paper's protocol) for VSamp (Algorithm 4), ESamp with exact
per-edge counts (Algorithm 5), ESamp with the fast per-edge estimate
(Algorithm 7, 1,000 repetitions), WSamp (Algorithm 6) and ESpar (Algorithm 8).

    python -m paper_1801_00338_gb300.samplers_eval [--small]

For each estimator: the variance of one draw (exact from the local counts for
VSamp and both ESamp forms, Lemma 4 / the ESamp lemma with the binomial term
of Algorithm 7; empirical for WSamp and ESpar), the draws needed for a 1%
median relative error (normal approximation: 0.6745 sd), the GPU time per
draw from one long call, the time to 1% that these give, and the median
relative error actually measured over 30 trials at that draw count (draw
counts capped by a time budget).  Prints one JSON object.
"""
from __future__ import annotations

import json
import math
import sys
import time

import numpy as np

from . import bfc, synth

Z50 = 0.6744897501960817  # median of |N(0, 1)|


def draws_for(var1: float, B: float, rel: float = 0.01) -> int:
    return max(1, int(math.ceil((Z50 / rel) ** 2 * var1 / (B * B))))


def _timed(fn):
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = fn()
    torch.cuda.synchronize()
    return out, time.perf_counter() - t0


def run(g, budget_s: float = 60.0, reps: int = 1000, p_espar: float = 0.05) -> dict:
    import torch
    out = {"graph": {"nU": g.nU, "nV": g.nV, "m": g.m}}
    with bfc.Graph(g.u, g.v, g.nU, g.nV) as G:
        (B, side), t_exact = _timed(lambda: G.exact(hub_mma=True))
        (B, side), t_exact = _timed(lambda: G.exact(hub_mma=True))
        out["exact"] = {"B": int(B), "s": t_exact}
        lU, lV, le, _ = G.local_counts()
        n, m = g.nU + g.nV, g.m
        b = torch.cat([lU, lV]).to(torch.float64)
        be = le.to(torch.float64)
        # exact single-draw variances
        Bf = float(B)
        var = {"vsamp": (n / 16.0) * float((b * b).sum().item()) - Bf * Bf,
               "esamp": (m / 16.0) * float((be * be).sum().item()) - Bf * Bf}
        cu, cv = G.edges()
        dU = torch.bincount(cu.long(), minlength=g.nU).to(torch.float64)
        dV = torch.bincount(cv.long(), minlength=g.nV).to(torch.float64)
        dd = dU[cu.long()] * dV[cv.long()]
        var["esamp_fast"] = var["esamp"] + (m / 16.0) * float((be * dd - be * be).sum().item()) / reps
        del lU, lV, le, b, be, cu, cv, dd
        samplers = {
            "vsamp": lambda k, T, s: G.vsamp(k, T, s),
            "esamp": lambda k, T, s: G.esamp(k, T, s),
            "esamp_fast": lambda k, T, s: G.esamp(k, T, s, reps=reps),
            "wsamp": lambda k, T, s: G.wsamp(k, T, s),
        }
        res = {}
        for name, fn in samplers.items():
            r = {}
            # pilot: per-draw time (and the empirical variance where no exact one exists)
            k0, T0 = 4096, 64
            fn(256, 2, 1)
            est, dt = _timed(lambda: fn(k0, T0, 2))
            spd = dt / (k0 * T0)
            if name in var:
                r["var_single"] = var[name]
                r["var_kind"] = "exact"
                r["var_single_empirical"] = float(np.var(est, ddof=1) * k0)
            else:
                r["var_single"] = float(np.var(est, ddof=1) * k0)
                r["var_kind"] = "empirical (64 trials x 4096 draws)"
            kk = draws_for(r["var_single"], B)
            r["draws_1pct"] = kk
            # the check: 30 trials at kk draws, capped by the time budget
            k_run = int(max(1, min(kk, budget_s / (30 * spd))))
            est, dt = _timed(lambda: fn(k_run, 30, 3))
            r["draws_run"] = k_run
            r["s_per_draw"] = dt / (k_run * 30)
            r["time_1pct_s"] = kk * r["s_per_draw"]
            r["median_rel_err_30"] = float(np.median(np.abs(est - B) / B))
            r["expected_median_rel_err"] = Z50 * math.sqrt(r["var_single"] / k_run) / B
            res[name] = r
        # ESpar: one trial is one "draw"
        r = {"p": p_espar}
        G.espar(p_espar, 2, 1)
        (est, beta), dt = _timed(lambda: G.espar(p_espar, 30, 4))
        est = np.asarray(est, np.float64)
        r["s_per_trial"] = dt / 30
        r["var_single"] = float(np.var(est, ddof=1))
        r["var_kind"] = "empirical (30 trials)"
        kk = draws_for(r["var_single"], B)
        r["trials_1pct"] = kk
        r["time_1pct_s"] = kk * r["s_per_trial"]
        r["median_rel_err_single_trial"] = float(np.median(np.abs(est - B) / B))
        res["espar"] = r
        out["samplers"] = res
    return out


if __name__ == "__main__":
    if "--small" in sys.argv:
        g = synth.chung_lu_scaled(20_000, 100_000, 1_000_000, 2.1, 2.5, 2)
        print(json.dumps(run(g, budget_s=10.0)))
    else:
        print(json.dumps(run(synth.chung_lu_1m_5m(), budget_s=60.0)))
