"""The GPU estimators over 1,000 seeded trials: each mean lies within three
standard errors of the exact count, the standard error taken from the exact
single-trial variance the oracle derives from the paper's moment formulas
(ESpar: Lemma 8; ClrSpar: Lemma 9; ESamp and WSamp: the second moments over
the butterfly-pair types of Section 5), not from the sample."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1801_00338_gb300 import synth

pytestmark = pytest.mark.gpu
T = 1000


@pytest.fixture(scope="module")
def bfc():
    import torch
    assert torch.cuda.is_available()
    from paper_1801_00338_gb300 import build as B
    B.build()
    from paper_1801_00338_gb300 import bfc as mod
    mod.load()
    return mod


def _dense(nU, nV, p, seed):
    r = synth.uniform01(seed, 0, nU * nV).reshape(nU, nV)
    a, x = np.nonzero(r < p)
    return a.astype(np.uint32), x.astype(np.uint32)


def test_espar_1000_trials(bfc):
    u, v = synth.uniform_bipartite(10, 10, 45, 8)
    B, _ = O.exact(u, v, 10, 10)
    pairs = O.pair_types(u, v)
    p = 0.5
    with bfc.Graph(u, v, 10, 10) as G:
        est, beta = G.espar(p, T, 2024)
    for t in range(0, T, 97):  # the trials are the oracle's, draw for draw
        assert int(beta[t]) == O.espar_trial(u, v, 10, 10, p, 2024, t)[0]
    var = O.espar_variance(B, pairs, O.espar_threshold(p) / 4294967296.0)
    assert abs(np.mean(est) - B) <= 3 * math.sqrt(var / T)


def test_clrspar_1000_trials(bfc):
    nU, nV = 12, 14
    u, v = _dense(nU, nV, 0.45, 6)
    B, _ = O.exact(u, v, nU, nV)
    pairs = O.pair_types(u, v)
    N = 3
    with bfc.Graph(u, v, nU, nV) as G:
        est, beta = G.clrspar(N, T, 31)
    for t in range(0, T, 97):
        assert int(beta[t]) == O.clrspar_trial(u, v, nU, nV, N, 31, t)[0]
    var = O.clrspar_variance(B, pairs, N)
    assert abs(np.mean(est) - B) <= 3 * math.sqrt(var / T)


@pytest.mark.parametrize("reps", [0, 10])
def test_esamp_1000_trials(bfc, reps):
    nU, nV = 12, 14
    u, v = _dense(nU, nV, 0.45, 6)
    B, _ = O.exact(u, v, nU, nV)
    be = O.per_edge(u, v, nU, nV)
    dA = np.bincount(u, minlength=nU)[u]
    dX = np.bincount(v, minlength=nV)[v]
    k = 5
    with bfc.Graph(u, v, nU, nV) as G:
        est = G.esamp(k, T, 11, reps=reps)
    var = O.esamp_term_variance(be, dA, dX, reps) / k
    assert abs(np.mean(est) - B) <= 3 * math.sqrt(var / T)


def test_wsamp_1000_trials(bfc):
    nU, nV = 12, 13
    u, v = _dense(nU, nV, 0.4, 10)
    B, _ = O.exact(u, v, nU, nV)
    W = O.wedges(u, v, nU, nV)
    beta = np.array([w[3] for w in W], np.float64)
    var1 = len(W) / 16.0 * (beta * beta).sum() - B * B
    k = 5
    with bfc.Graph(u, v, nU, nV) as G:
        est = G.wsamp(k, T, 21)
    assert abs(np.mean(est) - B) <= 3 * math.sqrt(var1 / k / T)
