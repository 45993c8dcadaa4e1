"""(epsilon, delta) estimates from the sampling estimators.

Section 5.1 makes an (epsilon, delta) estimator from one that is unbiased:
average alpha independent instances, so that Chebyshev's inequality bounds
the chance of a miss by epsilon B to 1/32, then take the median of
O(log 1/delta) such averages.  The paper sizes alpha from variance bounds
that need B and the butterfly pair counts; here a pilot run estimates the
variance of one instance and B, `bfc_mom_sizes` turns them into alpha and an
odd number of groups, and the answer is the median of the group means
(`bfc_median_of_means`).  Every instance is drawn on the GPU by the
library's samplers; this module only chooses sizes.

Instances: one draw for VSamp / ESamp / ESamp with Algorithm 7 / WSamp (a
trial of k draws is the mean of k instances, so a trial of alpha draws is one
group mean), one trial for ESpar / ClrSpar.
"""
from __future__ import annotations

import numpy as np

from . import bfc

DRAW_METHODS = ("vsamp", "esamp", "esamp_fast", "wsamp")
TRIAL_METHODS = ("espar", "clrspar")


def _draws(G: "bfc.Graph", method: str, k: int, trials: int, seed: int, reps: int) -> np.ndarray:
    if method == "vsamp":
        return np.asarray(G.vsamp(k, trials, seed), np.float64)
    if method == "esamp":
        return np.asarray(G.esamp(k, trials, seed), np.float64)
    if method == "esamp_fast":
        return np.asarray(G.esamp(k, trials, seed, reps=reps), np.float64)
    if method == "wsamp":
        return np.asarray(G.wsamp(k, trials, seed), np.float64)
    raise ValueError(method)


def _trials(G: "bfc.Graph", method: str, trials: int, seed: int, p: float, colors: int) -> np.ndarray:
    if method == "espar":
        est, _ = G.espar(p, trials, seed)
    elif method == "clrspar":
        est, _ = G.clrspar(colors, trials, seed)
    else:
        raise ValueError(method)
    return np.asarray(est, np.float64)


def estimate(G: "bfc.Graph", method: str, epsilon: float, delta: float, seed: int = 0,
             pilot_draws: int = 4096, pilot_trials: int = 32, reps: int = 1000, p: float = 0.05,
             colors: int = 20) -> dict:
    """An (epsilon, delta) estimate of B with `method`.  Returns the estimate,
    the sizes used and the pilot's variance and mean."""
    if method in DRAW_METHODS:
        pilot = _draws(G, method, pilot_draws, pilot_trials, seed, reps)
        var1 = float(np.var(pilot, ddof=1)) * pilot_draws
    elif method in TRIAL_METHODS:
        pilot = _trials(G, method, pilot_trials, seed, p, colors)
        var1 = float(np.var(pilot, ddof=1))
    else:
        raise ValueError(f"unknown method {method!r}")
    B_pilot = float(np.mean(pilot))
    if B_pilot <= 0.0:
        return {"estimate": 0.0, "alpha": 0, "groups": 0, "var1": var1, "pilot_mean": B_pilot}
    alpha, groups = bfc.bfc_mom_sizes(var1, B_pilot, epsilon, delta)
    if method in DRAW_METHODS:
        means = _draws(G, method, alpha, groups, seed + 1, reps)   # one trial = one group mean
        est = bfc.bfc_median_of_means(means, groups)
    else:
        y = _trials(G, method, alpha * groups, seed + 1, p, colors)
        est = bfc.bfc_median_of_means(y, groups)
    return {"estimate": est, "alpha": alpha, "groups": groups, "var1": var1, "pilot_mean": B_pilot}
