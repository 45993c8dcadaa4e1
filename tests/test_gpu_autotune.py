"""Scheduling settings (bfc_tuning) and the autotuner on the GPU: every
setting gives the oracle's counts bit for bit, and the autotuner keeps one
of them and caches it."""
import numpy as np
import pytest

import oracle as O
from paper_1801_00338_gb300 import synth

pytestmark = pytest.mark.gpu

NO_HUBS = 0xFFFFFFFF
NO_FLAT = 0xFFFFFFFF
NO_HL = 0xFFFFFFFF
# extreme and typical settings: every vertex past the warp class in the large
# windows or the big class (small_max_segs = 1), almost no warp class
# (warp_max_wedges = 1), hub blocks of one tile and of none, the densest
# column threshold, whole-row local counts, and the flat expansion of
# single-window vertices never or always taken, and the heavy-light split
# never, for almost no vertex, or up to a middle limit
TUNINGS = [
    {},
    {"small_max_segs": 1},
    {"small_max_segs": 64, "warp_max_wedges": 128},
    {"warp_max_wedges": 1},
    {"hubs": 128, "tau": 2},
    {"hubs": 1024},
    {"hubs": NO_HUBS},
    {"local_sweep": 1, "small_max_segs": 100},
    {"flat_max_avg": NO_FLAT},
    {"flat_max_avg": 0xFFFFFFFE},
    {"flat_max_avg": 0xFFFFFFFE, "local_sweep": 1},
    {"hl_max_light": NO_HL},
    {"hl_max_light": 1},
    {"hl_max_light": 300, "small_max_segs": 1},
    {"hl_max_light": NO_HL, "flat_max_avg": NO_FLAT},
]


@pytest.fixture(scope="module")
def bfc():
    import torch
    assert torch.cuda.is_available()
    from paper_1801_00338_gb300 import build as B
    B.build()
    from paper_1801_00338_gb300 import bfc as mod
    mod.load()
    return mod


def u64(t):
    return t.cpu().numpy().view(np.uint64)


@pytest.fixture(scope="module")
def skewed():
    """120k x 30k Chung-Lu graph whose start vertices span several rank windows
    and every kernel class."""
    g = synth.chung_lu_scaled(120_000, 30_000, 600_000, 2.1, 2.5, 31)
    oB, _ = O.exact(g.u, g.v, g.nU, g.nV)
    oU, oV = O.per_vertex(g.u, g.v, g.nU, g.nV)
    return g, oB, oU, oV


@pytest.mark.parametrize("tuning", TUNINGS, ids=[str(i) for i in range(len(TUNINGS))])
def test_counts_do_not_depend_on_the_settings(bfc, skewed, tuning):
    g, oB, oU, oV = skewed
    with bfc.Graph(g.u, g.v, g.nU, g.nV) as G:
        G.set_tuning(tuning)
        got = G.tuning()
        for k, val in tuning.items():
            assert got[k] == val
        assert G.exact(hub_mma=True)[0] == oB
        assert G.exact()[0] == oB
        bU, bV, be, B = G.local_counts()
        assert B == oB
        assert np.array_equal(u64(bU), oU) and np.array_equal(u64(bV), oV)
        be = u64(be)
        assert int(be.sum()) == 4 * oB
        idx = np.arange(0, g.m, 4099, dtype=np.uint64)
        cu, cv = G.edges()
        want = O.per_edge_list(cu.cpu().numpy().astype(np.uint32), cv.cpu().numpy().astype(np.uint32),
                               g.nU, g.nV, idx)
        assert np.array_equal(be[idx.astype(np.int64)], want)
        # sparsification trials classify their kept subgraphs with the same limits
        _, beta = G.espar(0.5, 2, 77)
        for t in range(2):
            assert int(beta[t]) == O.espar_trial(g.u, g.v, g.nU, g.nV, 0.5, 77, t)[0]


def test_changing_the_settings_on_a_built_plan(bfc, skewed):
    """The rank layout is kept and only the classes are redone, in both directions."""
    g, oB, oU, oV = skewed
    with bfc.Graph(g.u, g.v, g.nU, g.nV) as G:
        assert G.exact()[0] == oB
        s0 = G.plan_stats(0)
        G.set_tuning({"small_max_segs": 1, "warp_max_wedges": 1})
        assert G.exact()[0] == oB
        s1 = G.plan_stats(0)
        assert s1["count"]["warp"] < s0["count"]["warp"]
        assert sum(s1["count"][c] for c in ("s2", "s4", "s8", "s6", "s5")) == 0
        G.set_tuning(None)
        assert G.exact()[0] == oB
        assert G.plan_stats(0)["count"] == s0["count"]
        bU, bV, B = G.per_vertex()
        assert B == oB and np.array_equal(u64(bU), oU) and np.array_equal(u64(bV), oV)


def test_invalid_settings_are_rejected(bfc, skewed):
    g = synth.uniform_small(1)
    with bfc.Graph(g.u, g.v, g.nU, g.nV) as G:
        for bad in ({"warp_max_wedges": 513}, {"small_max_segs": 600}, {"hubs": 100}, {"hubs": 32768},
                    {"tau": 1}, {"local_sweep": 2}):
            with pytest.raises(bfc.BfcError) as e:
                G.set_tuning(bad)
            assert e.value.code == -1
        with pytest.raises(ValueError):
            G.set_tuning({"no_such_field": 1})
        # a hub count larger than the start side falls back to the whole tiles it has
        G.set_tuning({"hubs": 16384})
        assert G.exact(hub_mma=True)[0] == O.exact(g.u, g.v, g.nU, g.nV)[0]


def test_autotune_keeps_a_setting_with_the_same_counts_and_caches_it(bfc, skewed, tmp_path):
    from paper_1801_00338_gb300 import autotune as A
    g, oB, oU, oV = skewed
    path = str(tmp_path / "tuning.json")
    with bfc.Graph(g.u, g.v, g.nU, g.nV) as G:
        r = A.autotune(G, ("exact", "local"), cache_path=path, reps=2)
        assert r.source == "search"
        assert r.counts[0] == oB and r.counts[1] == oB
        assert r.counts[2] == int(oU.sum()) == 2 * oB
        assert r.ms <= r.default_ms
        assert len(r.tried) >= 8
        assert G.tuning() == r.tuning
        assert G.exact(hub_mma=True)[0] == oB
    with bfc.Graph(g.u, g.v, g.nU, g.nV) as G:
        r2 = A.autotune(G, ("exact", "local"), cache_path=path, reps=1)
        assert r2.source == "cache" and r2.tuning == r.tuning
