"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Counts are integers: every comparison is exact (bit for bit).
"""
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


def u64(t):
    return t.cpu().numpy().view(np.uint64)


def check_all(bfc, u, v, nU, nV, per_edge=True, sides=(None, "U", "V")):
    oB, oside = O.exact(u, v, nU, nV)
    with bfc.Graph(u, v, nU, nV) as G:
        for side in sides:
            B, s = G.exact(side)
            assert B == oB, (side, B, oB)
            if side is None:
                assert s == oside
        oU, oV = O.per_vertex(u, v, nU, nV)
        for whole in (False, True):
            bU, bV, B2 = G.per_vertex(whole_rows=whole)
            assert B2 == oB
            assert np.array_equal(u64(bU), oU)
            assert np.array_equal(u64(bV), oV)
        if per_edge:
            can = O.canonical_ids(u, v, nU, nV)
            oe = O.per_edge(u, v, nU, nV)
            for whole in (False, True):
                be, B3 = G.per_edge(whole_rows=whole)
                assert B3 == oB
                assert np.array_equal(u64(be)[can], oe)
            for whole in (False, True):
                lU, lV, le, B4 = G.local_counts(whole_rows=whole)
                assert B4 == oB
                assert np.array_equal(u64(lU), oU) and np.array_equal(u64(lV), oV)
                assert np.array_equal(u64(le)[can], oe)
    return oB


def test_uniform_2000x3000(bfc):
    g = synth.uniform_small(1)
    assert check_all(bfc, g.u, g.v, g.nU, g.nV) > 0


def test_tiny_random_graphs(bfc):
    rs = synth.uniform01(21, 0, 3 * 150).reshape(150, 3)
    for i in range(150):
        nU = 1 + int(rs[i, 0] * 12)
        nV = 1 + int(rs[i, 1] * 12)
        m = int(rs[i, 2] * nU * nV)
        if m == 0:
            continue
        u, v = synth.uniform_bipartite(nU, nV, m, 500 + i)
        check_all(bfc, u, v, nU, nV)


@pytest.mark.parametrize("a,b", [(2, 2), (3, 40), (40, 3), (700, 30), (10000, 10)])
def test_bicliques(bfc, a, b):
    u, v = synth.complete_bipartite(a, b)
    C2 = lambda k: k * (k - 1) // 2
    with bfc.Graph(u, v, a, b) as G:
        for side in (None, "U", "V"):
            assert G.exact(side)[0] == C2(a) * C2(b)
        bU, bV, _ = G.per_vertex()
        assert (u64(bU) == (a - 1) * C2(b)).all() and (u64(bV) == (b - 1) * C2(a)).all()
        if a * b <= 30000:
            be, _ = G.per_edge()
            assert (u64(be) == (a - 1) * (b - 1)).all()


def test_table1_biclique_side_and_count(bfc):
    """Table 1 row 1: (10^4, 10)-biclique, B = 2,249,775,000; Algorithm 1 starts from R (= V)."""
    u, v = synth.complete_bipartite(10000, 10)
    with bfc.Graph(u, v, 10000, 10) as G:
        assert G.stats["sq_u"] == 10 ** 6 and G.stats["sq_v"] == 10 ** 9
        assert G.exact() == (2249775000, 1)


def test_skewed_graph_spanning_several_rank_windows(bfc):
    """|U| = 120k start vertices (three 48k-rank windows) with a power-law skew, so the
    warp and CTA classes both run and CTA vertices walk several windows."""
    g = synth.chung_lu_scaled(120_000, 30_000, 600_000, 2.1, 2.5, 31)
    check_all(bfc, g.u, g.v, g.nU, g.nV, per_edge=False)
    with bfc.Graph(g.u, g.v, g.nU, g.nV) as G:
        be, B = G.per_edge()
        be = u64(be)
        assert int(be.sum()) == 4 * B
        cu, cv = G.edges()
        cu = cu.cpu().numpy().astype(np.uint32)
        cv = cv.cpu().numpy().astype(np.uint32)
        idx = np.arange(0, g.m, 997, dtype=np.uint64)
        want = O.per_edge_list(cu, cv, g.nU, g.nV, idx)
        assert np.array_equal(be[idx.astype(np.int64)], want)


def test_medium_chung_lu_per_edge(bfc):
    g = synth.chung_lu_scaled(3000, 9000, 40_000, 2.1, 2.4, 5)
    check_all(bfc, g.u, g.v, g.nU, g.nV)


def test_empty_and_degenerate(bfc):
    z = np.zeros(0, np.uint32)
    with bfc.Graph(z, z, 5, 7) as G:
        assert G.exact()[0] == 0
        bU, bV, B = G.per_vertex()
        assert B == 0 and int(u64(bU).sum()) == 0 and int(u64(bV).sum()) == 0
    one = np.array([0], np.uint32)
    with bfc.Graph(one, one, 1, 1) as G:
        assert G.exact()[0] == 0
    star_u = np.zeros(50, np.uint32)
    star_v = np.arange(50, dtype=np.uint32)
    with bfc.Graph(star_u, star_v, 1, 50) as G:
        assert G.exact()[0] == 0 and G.exact("V")[0] == 0


def test_input_errors(bfc):
    u = np.array([0, 1, 0], np.uint32)
    v = np.array([0, 1, 0], np.uint32)
    with pytest.raises(bfc.BfcError) as e:
        bfc.Graph(u, v, 2, 2)
    assert e.value.code == -3
    with bfc.Graph(u, v, 2, 2, dedup=True) as G:
        assert G.m == 2 and G.exact()[0] == 0
    with pytest.raises(bfc.BfcError) as e:
        bfc.Graph(np.array([2], np.uint32), np.array([0], np.uint32), 2, 2)
    assert e.value.code == -2


def test_dedup_matches_oracle_on_deduplicated_edges(bfc):
    u, v = synth.uniform_bipartite(50, 60, 900, 4)
    uu = np.concatenate([u, u[:300]])
    vv = np.concatenate([v, v[:300]])
    with bfc.Graph(uu, vv, 50, 60, dedup=True) as G:
        assert G.m == 900
        assert G.exact()[0] == O.exact(u, v, 50, 60)[0]


def test_device_input(bfc):
    import torch
    g = synth.uniform_small(3)
    du = torch.from_numpy(g.u.astype(np.int32)).cuda()
    dv = torch.from_numpy(g.v.astype(np.int32)).cuda()
    with bfc.Graph(du, dv, g.nU, g.nV) as G:
        assert G.exact()[0] == O.exact(g.u, g.v, g.nU, g.nV)[0]


def test_canonical_edges(bfc):
    g = synth.uniform_small(4)
    with bfc.Graph(g.u, g.v, g.nU, g.nV) as G:
        cu, cv = G.edges()
    key = g.u.astype(np.uint64) * np.uint64(g.nV) + g.v
    srt = np.sort(key)
    got = cu.cpu().numpy().astype(np.uint64) * np.uint64(g.nV) + cv.cpu().numpy().astype(np.uint64)
    assert np.array_equal(got, srt)


@pytest.mark.parametrize("side_stream", [False, True])
def test_espar_trials_match_oracle(bfc, side_stream):
    """Trial by trial; on a side stream the trials after the first replay a recorded CUDA graph."""
    import torch
    g = synth.uniform_small(1)
    st = torch.cuda.Stream() if side_stream else None
    with bfc.Graph(g.u, g.v, g.nU, g.nV) as G:
        est, beta = G.espar(0.3, 6, 1234, stream=st)
    for t in range(6):
        ob, oe = O.espar_trial(g.u, g.v, g.nU, g.nV, 0.3, 1234, t)
        assert int(beta[t]) == ob
        assert est[t] == oe


def test_espar_on_multi_window_graph_side_stream(bfc):
    import torch
    g = synth.chung_lu_scaled(120_000, 30_000, 600_000, 2.1, 2.5, 31)
    st = torch.cuda.Stream()
    with bfc.Graph(g.u, g.v, g.nU, g.nV) as G:
        est, beta = G.espar(0.5, 3, 77, stream=st)
        est2, beta2 = G.clrspar(2, 3, 78, stream=st)
    for t in range(3):
        assert int(beta[t]) == O.espar_trial(g.u, g.v, g.nU, g.nV, 0.5, 77, t)[0]
        assert int(beta2[t]) == O.clrspar_trial(g.u, g.v, g.nU, g.nV, 2, 78, t)[0]


@pytest.mark.parametrize("side_stream", [False, True])
def test_clrspar_trials_match_oracle(bfc, side_stream):
    import torch
    g = synth.chung_lu_scaled(3000, 9000, 40_000, 2.1, 2.4, 5)
    st = torch.cuda.Stream() if side_stream else None
    with bfc.Graph(g.u, g.v, g.nU, g.nV) as G:
        est, beta = G.clrspar(3, 5, 99, stream=st)
    for t in range(5):
        ob, oe = O.clrspar_trial(g.u, g.v, g.nU, g.nV, 3, 99, t)
        assert int(beta[t]) == ob
        assert est[t] == oe


@pytest.mark.parametrize("side_stream", [False, True])
def test_many_sparse_trials_match_oracle(bfc, side_stream):
    """70 ESpar trials at p = 0.05 and 70 ClrSpar trials with 20 colours (the
    batched estimators' settings), trial by trial: the persistent launch takes
    its work in chunks of 32 trials, so 70 spans a ragged third chunk; on a
    side stream the launches are recorded into one CUDA graph."""
    import torch
    g = synth.chung_lu_scaled(20_000, 40_000, 300_000, 2.0, 2.3, 3)
    st = torch.cuda.Stream() if side_stream else None
    with bfc.Graph(g.u, g.v, g.nU, g.nV) as G:
        _, beta = G.espar(0.05, 70, 2024, stream=st)
        _, beta2 = G.clrspar(20, 70, 2025, stream=st)
    for t in range(70):
        assert int(beta[t]) == O.espar_trial(g.u, g.v, g.nU, g.nV, 0.05, 2024, t)[0], t
        assert int(beta2[t]) == O.clrspar_trial(g.u, g.v, g.nU, g.nV, 20, 2025, t)[0], t


def test_dense_trials_take_the_heavy_path(bfc):
    """Keep probability 0.9 on a skewed graph: most (start vertex, trial) pairs
    overflow the per-warp tables and are counted from the heavy list by whole
    CTAs with global tables; every trial still equals the oracle's."""
    g = synth.chung_lu_scaled(30_000, 8_000, 200_000, 2.1, 2.5, 41)
    with bfc.Graph(g.u, g.v, g.nU, g.nV) as G:
        _, beta = G.espar(0.9, 5, 555)
        _, beta2 = G.clrspar(1, 2, 556)
    B = O.exact(g.u, g.v, g.nU, g.nV)[0]
    for t in range(5):
        assert int(beta[t]) == O.espar_trial(g.u, g.v, g.nU, g.nV, 0.9, 555, t)[0], t
    assert [int(b) for b in beta2] == [B, B]  # one colour keeps every edge


def _vsamp_check(bfc, g, k, trials, seed, weights=None):
    import torch
    with bfc.Graph(g.u, g.v, g.nU, g.nV) as G:
        prop = bfc.bfc_proposal_from_weights(G.h, weights) if weights is not None else None
        try:
            est, drawn, bd = G.vsamp(k, trials, seed, proposal=prop, want_draws=True)
        finally:
            if prop:
                bfc.bfc_proposal_free(prop)
        drawn = u64(drawn).reshape(trials, k)
        bd = u64(bd).reshape(trials, k)
    for t in range(trials):
        oe, od, ob = O.vsamp_trial(g.u, g.v, g.nU, g.nV, k, seed, t, weights=weights)
        assert np.array_equal(drawn[t], od)
        assert np.array_equal(bd[t], ob)
        assert est[t] == pytest.approx(oe, rel=1e-12, abs=0.0)


def test_vsamp_uniform_matches_oracle(bfc):
    g = synth.chung_lu_scaled(3000, 9000, 40_000, 2.1, 2.4, 5)
    _vsamp_check(bfc, g, 300, 4, 77)


def test_vsamp_weighted_matches_oracle(bfc):
    g = synth.chung_lu_scaled(3000, 9000, 40_000, 2.1, 2.4, 6)
    n = g.nU + g.nV
    w = (synth.splitmix64(9, 0, n) >> np.uint64(44)).astype(np.uint32)
    _vsamp_check(bfc, g, 500, 3, 5, weights=w)


def test_vsamp_on_multi_window_graph(bfc):
    """Draws that land on CTA-class vertices walk every rank window (whole midpoint rows)."""
    g = synth.chung_lu_scaled(120_000, 30_000, 600_000, 2.1, 2.5, 31)
    _vsamp_check(bfc, g, 64, 2, 3)


def test_batched_uneven_graphs_match_oracle(bfc):
    """Many graphs of uneven size and skew in one pass; each graph's B and start side."""
    params = synth.uneven_batch_params(48, 17, m_lo=50, m_hi=30_000)
    graphs = []
    for i, (nU, nV, m, gamma) in enumerate(params):
        u, v = synth.chung_lu_bipartite(nU, nV, m, gamma, gamma, 300 + i)
        graphs.append((u, v, nU, nV))
    graphs.append(tuple(list(synth.complete_bipartite(30, 4)) + [30, 4]))   # starts from V
    graphs.append((np.zeros(0, np.uint32), np.zeros(0, np.uint32), 3, 5))   # no edges
    B, side = bfc.bfc_exact_batch(graphs)
    for (u, v, nU, nV), b, sd in zip(graphs, B, side):
        ob, os_ = O.exact(u, v, nU, nV)
        assert int(b) == ob and int(sd) == os_


def test_batched_graphs_spanning_rank_windows(bfc):
    """Graphs large enough that a start vertex's targets would span several
    counter windows of the union, each counted within its own rank range."""
    params = synth.uneven_batch_params(96, 23, m_lo=2_000, m_hi=200_000)
    graphs = []
    for i, (nU, nV, m, gamma) in enumerate(params):
        u, v = synth.chung_lu_bipartite(nU, nV, m, gamma, gamma, 900 + i)
        graphs.append((u, v, nU, nV))
    B, side = bfc.bfc_exact_batch(graphs)
    for (u, v, nU, nV), b, sd in zip(graphs, B, side):
        ob, os_ = O.exact(u, v, nU, nV)
        assert int(b) == ob and int(sd) == os_


def _rows(u, v, nU, nV):
    """Host CSR of both sides: U rows ascending in v (canonical order), V rows
    ascending in u, and the canonical id of each V-row entry."""
    order = np.lexsort((v, u))
    cu, cv = u[order].astype(np.int64), v[order].astype(np.int64)
    offU = np.zeros(nU + 1, np.int64)
    np.add.at(offU, cu + 1, 1)
    offU = np.cumsum(offU)
    vo = np.lexsort((cu, cv))
    offV = np.zeros(nV + 1, np.int64)
    np.add.at(offV, cv + 1, 1)
    offV = np.cumsum(offV)
    return offU, cv.astype(np.int32), offV, cu[vo].astype(np.int32), vo.astype(np.int32)


def test_graph_from_csr_matches_edge_list(bfc):
    import torch
    g = synth.chung_lu_scaled(3000, 9000, 60_000, 2.1, 2.4, 5)
    offU, nbrU, offV, nbrV, eidV = _rows(g.u, g.v, g.nU, g.nV)
    t = [torch.from_numpy(a).cuda() for a in (offU, nbrU, offV, nbrV, eidV)]
    oB, _ = O.exact(g.u, g.v, g.nU, g.nV)
    oU, oV = O.per_vertex(g.u, g.v, g.nU, g.nV)
    with bfc.Graph(g.u, g.v, g.nU, g.nV) as G0:
        e0, _ = G0.per_edge()
        for eid in (None, t[4]):
            G = bfc.Graph.from_csr(t[0], t[1], g.nU, t[2], t[3], g.nV, eidV=eid)
            try:
                assert G.stats == G0.stats
                assert G.exact()[0] == oB and G.exact(hub_mma=True)[0] == oB
                bU, bV, B = G.per_vertex()
                assert B == oB and np.array_equal(u64(bU), oU) and np.array_equal(u64(bV), oV)
                be, _ = G.per_edge()
                assert np.array_equal(u64(be), u64(e0))   # same canonical order
            finally:
                G.close()


def test_graph_from_csr_rejects_malformed_rows(bfc):
    import torch
    u, v = synth.uniform_bipartite(60, 50, 600, 3)
    offU, nbrU, offV, nbrV, eidV = _rows(u, v, 60, 50)

    def build(oU=offU, nU_=nbrU, oV=offV, nV_=nbrV, eid=None, nu=60, nv=50):
        t = [torch.from_numpy(np.ascontiguousarray(a)).cuda() for a in (oU, nU_, oV, nV_)]
        e = torch.from_numpy(np.ascontiguousarray(eid)).cuda() if eid is not None else None
        bfc.bfc_graph_free(bfc.bfc_graph_from_csr(t[0], t[1], nu, t[2], t[3], nv, e))

    build()
    build(eid=eidV)
    a = int(np.argmax(np.diff(offU) >= 2))          # a U row with two entries: swap them
    bad = nbrU.copy()
    bad[offU[a]], bad[offU[a] + 1] = bad[offU[a] + 1], bad[offU[a]]
    cases = [(dict(nU_=bad), -1),                      # row not ascending
             (dict(nU_=np.where(np.arange(nbrU.size) == 0, 50, nbrU).astype(np.int32)), -2),  # V id out of range
             (dict(oV=np.concatenate([offV[:-1], [offV[-1] - 1]])), -1),   # the sides disagree on m
             (dict(eid=np.roll(eidV, 1)), -1)]          # inconsistent edge ids
    for kw, code in cases:
        with pytest.raises(bfc.BfcError) as ei:
            build(**kw)
        assert ei.value.code == code, kw
