"""Edge sampling (Algorithm 5, exact b_e per draw or Algorithm 7's fast
estimate) and wedge sampling (Algorithm 6) on the GPU against the oracle:
the drawn edges / centres and the integer value of every draw are compared
bit for bit; the per-trial estimates within floating-point summation order."""
import numpy as np
import pytest

import oracle as O
from paper_1801_00338_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bfc():
    import torch
    assert torch.cuda.is_available()
    from paper_1801_00338_gb300 import build as B
    B.build()
    from paper_1801_00338_gb300 import bfc as mod
    mod.load()
    return mod


def dense(nU, nV, p, seed):
    r = synth.uniform01(seed, 0, nU * nV).reshape(nU, nV)
    a, x = np.nonzero(r < p)
    return a.astype(np.uint32), x.astype(np.uint32)


GRAPHS = {
    "dense_40x50": lambda: (*dense(40, 50, 0.3, 3), 40, 50),
    "uniform_2000x3000": lambda: (lambda g: (g.u, g.v, g.nU, g.nV))(synth.uniform_small(1)),
    "chung_lu_multiwindow": lambda: (lambda g: (g.u, g.v, g.nU, g.nV))(
        synth.chung_lu_scaled(120000, 30000, 600000, 2.1, 2.5, 31)),
}


def u64(t):
    return t.cpu().numpy().view(np.uint64)


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("reps", [0, 1, 7, 1000])
def test_esamp_matches_oracle(bfc, name, reps):
    u, v, nU, nV = GRAPHS[name]()
    k, trials, seed = 300, 3, 41
    with bfc.Graph(u, v, nU, nV) as G:
        est, ed, vd = G.esamp(k, trials, seed, reps=reps, want_draws=True)
    ed, vd = u64(ed).reshape(trials, k), u64(vd).reshape(trials, k)
    for t in range(trials):
        oe, oed, ovd = O.esamp_trial(u, v, nU, nV, k, reps, seed, t)
        assert np.array_equal(ed[t], oed), t
        assert np.array_equal(vd[t], ovd), t
        assert est[t] == pytest.approx(oe, rel=1e-12, abs=1e-9)


def test_esamp_exact_uses_both_probe_paths(bfc):
    """On the skewed graph some draws probe a neighbourhood larger than the
    shared hash (binary search in the row) and some a smaller one: both give
    the oracle's b_e (checked above); here check both paths were taken."""
    u, v, nU, nV = GRAPHS["chung_lu_multiwindow"]()
    dU = np.bincount(u, minlength=nU).astype(np.int64)
    dV = np.bincount(v, minlength=nV).astype(np.int64)
    sU = np.zeros(nU, np.int64)
    np.add.at(sU, u, dV[v])   # sum of d_x over a's row: cost of walking Gamma_a's rows
    sV = np.zeros(nV, np.int64)
    np.add.at(sV, v, dU[u])   # cost of walking Gamma_x's rows
    _, ed, _ = O.esamp_trial(u, v, nU, nV, 300, 0, 41, 0)
    order = np.lexsort((v, u))
    cu, cv = u[order], v[order]
    a, x = cu[ed.astype(np.int64)], cv[ed.astype(np.int64)]
    probe = np.where(sV[x] <= sU[a], dU[a], dV[x])   # the probe set is the other neighbourhood
    assert (probe > 4096).any() and (probe <= 4096).any()


@pytest.mark.parametrize("name", list(GRAPHS))
def test_wsamp_matches_oracle(bfc, name):
    u, v, nU, nV = GRAPHS[name]()
    k, trials, seed = 400, 3, 17
    with bfc.Graph(u, v, nU, nV) as G:
        est, cd, bd = G.wsamp(k, trials, seed, want_draws=True)
    cd, bd = u64(cd).reshape(trials, k), u64(bd).reshape(trials, k)
    for t in range(trials):
        oe, ocd, obd = O.wsamp_trial(u, v, nU, nV, k, seed, t)
        assert np.array_equal(cd[t], ocd), t
        assert np.array_equal(bd[t], obd), t
        assert est[t] == pytest.approx(oe, rel=1e-12, abs=1e-9)


def test_samplers_unbiased_on_medium_graph(bfc):
    """Means of many GPU trials land within 4 standard errors of the exact B
    (the oracle's count), for ESamp exact, ESamp with Algorithm 7 and WSamp."""
    g = synth.chung_lu_scaled(3000, 9000, 60_000, 2.1, 2.4, 5)
    B, _ = O.exact(g.u, g.v, g.nU, g.nV)
    with bfc.Graph(g.u, g.v, g.nU, g.nV) as G:
        for est in (G.esamp(200, 400, 5), G.esamp(200, 400, 6, reps=64), G.wsamp(400, 400, 7)):
            se = est.std(ddof=1) / np.sqrt(est.size)
            assert abs(est.mean() - B) <= 4 * se


def test_edge_cases(bfc):
    # a graph without butterflies: every draw is 0
    n = 300
    u = np.arange(n, dtype=np.uint32)
    v = np.arange(n, dtype=np.uint32)
    with bfc.Graph(u, v, n, n) as G:
        assert (G.esamp(50, 2, 1) == 0).all()
        assert (G.esamp(50, 2, 1, reps=10) == 0).all()
        with pytest.raises(bfc.BfcError):   # no wedge to draw
            G.wsamp(10, 1, 1)
        assert (G.esamp(0, 3, 1) == 0).all()   # no draws
    # K_{5,4} (B = C(5,2) C(4,2) = 60): every edge lies in (5-1)(4-1) = 12
    # butterflies, so every ESamp term is 12 m / 4 = B; a wedge centred on U
    # (endpoints in V) has 5 - 1 = 4 butterflies, one centred on V has 3
    u, v = synth.complete_bipartite(5, 4)
    with bfc.Graph(u, v, 5, 4) as G:
        est, _, vd = G.esamp(40, 2, 3, want_draws=True)
        assert (u64(vd) == 12).all() and np.allclose(est, 60.0)
        est, cd, bd = G.wsamp(40, 2, 3, want_draws=True)
        cd, bd = u64(cd), u64(bd)
        assert np.array_equal(bd, np.where(cd < 5, 4, 3))


def test_median_of_means_estimates_meet_epsilon(bfc):
    """(epsilon, delta) estimates (pilot-sized alpha and groups, median of
    group means) from each sampler land within epsilon B of the oracle's B in
    at least 1 - delta of the seeds (the sizes leave a wide margin)."""
    from paper_1801_00338_gb300 import mom
    g = synth.chung_lu_scaled(3000, 9000, 60_000, 2.1, 2.4, 5)
    B, _ = O.exact(g.u, g.v, g.nU, g.nV)
    eps, delta, runs = 0.1, 0.2, 10
    with bfc.Graph(g.u, g.v, g.nU, g.nV) as G:
        for method in ("vsamp", "esamp", "esamp_fast", "wsamp", "espar"):
            miss = 0
            for seed in range(runs):
                r = mom.estimate(G, method, eps, delta, seed=100 * seed, reps=64, p=0.3)
                assert r["groups"] % 2 == 1 and r["alpha"] >= 1
                miss += abs(r["estimate"] - B) > eps * B
            assert miss <= delta * runs, (method, miss)
