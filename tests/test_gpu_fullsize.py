"""The 1M x 5M, 50M-edge Chung-Lu workload (exponents 2.1 / 2.5), in the launch
configuration the benchmark times: sampled outputs against the oracle computed
one by one, and identities that hold at any size."""
import numpy as np
import pytest

import oracle as O
from paper_1801_00338_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def big():
    import torch
    assert torch.cuda.is_available()
    from paper_1801_00338_gb300 import build as B
    B.build()
    from paper_1801_00338_gb300 import bfc
    g = synth.chung_lu_1m_5m()
    G = bfc.Graph(g.u, g.v, g.nU, g.nV)
    yield g, G
    G.close()


def u64(t):
    return t.cpu().numpy().view(np.uint64)


def test_identities_and_sampled_vertices(big):
    g, G = big
    B, side = G.exact()
    assert side == 0  # sum_U d^2 > sum_V d^2: U starts, wedges are centred on V
    bU, bV, B2 = G.per_vertex()
    assert B2 == B
    bU, bV = u64(bU), u64(bV)
    oU2, oV2, _ = G.per_vertex(whole_rows=True)
    assert np.array_equal(u64(oU2), bU) and np.array_equal(u64(oV2), bV)
    assert int(bU.sum()) == 2 * B and int(bV.sum()) == 2 * B
    dU = np.bincount(g.u, minlength=g.nU)
    # sample: the 20 highest-degree vertices and 180 spread over the rest, each side
    idsU = np.unique(np.concatenate([np.argsort(dU)[-20:], np.arange(0, g.nU, g.nU // 180)])).astype(np.uint32)
    dV = np.bincount(g.v, minlength=g.nV)
    idsV = np.unique(np.concatenate([np.argsort(dV)[-20:], np.arange(0, g.nV, g.nV // 180)])).astype(np.uint32)
    assert np.array_equal(bU[idsU], O.per_vertex_list(g.u, g.v, g.nU, g.nV, 0, idsU))
    assert np.array_equal(bV[idsV], O.per_vertex_list(g.u, g.v, g.nU, g.nV, 1, idsV))


def test_per_edge_identities_and_samples(big):
    g, G = big
    B, _ = G.exact()
    be, B3 = G.per_edge()
    assert B3 == B
    be = u64(be)
    # the whole-row sweep and the combined call agree element by element
    be2, _ = G.per_edge(whole_rows=True)
    assert np.array_equal(u64(be2), be)
    lU, lV, le, B4 = G.local_counts()
    assert B4 == B and np.array_equal(u64(le), be)
    assert int(be.sum()) == 4 * B
    cu, cv = G.edges()
    cu = cu.cpu().numpy().astype(np.uint32)
    cv = cv.cpu().numpy().astype(np.uint32)
    # b_x = 1/2 sum of b_e over x's edges, on the V side
    bU, bV, _ = G.per_vertex()
    sV = np.zeros(g.nV, np.uint64)
    np.add.at(sV, cv, be)
    assert np.array_equal(sV, 2 * u64(bV))
    idx = np.arange(0, g.m, g.m // 150, dtype=np.uint64)
    assert np.array_equal(be[idx.astype(np.int64)], O.per_edge_list(cu, cv, g.nU, g.nV, idx))


def test_start_side_invariance(big):
    g, G = big
    B, _ = G.exact()
    assert G.exact("U")[0] == B
    assert G.exact("V")[0] == B  # 35x the wedges (centred on U), same count


def test_hub_block_same_count(big):
    """The tensor-core hub block in the benchmark's configuration (automatic
    hub set; and the top 16,384 U ranks) gives the walk's count."""
    g, G = big
    B, _ = G.exact()
    Bh, side, st = G.exact_hub()
    assert side == 0 and 0 < st["hubs"] <= 16384 and st["hubs"] % 128 == 0
    assert 0 < st["K"] <= 65536 and st["light_pairs"] > 0
    assert Bh == B
    Bh, _, st = G.exact_hub(hubs=16384)
    assert Bh == B and st["hubs"] == 16384
    assert G.exact(hub_mma=True)[0] == B


def test_samplers_draws_match_oracle(big):
    """ESamp (exact and with Algorithm 7, 1,000 repetitions) and WSamp on the
    full graph: every drawn edge / centre and the integer value of every draw
    equal the oracle's, computed draw by draw."""
    g, G = big
    for reps, k in ((0, 60), (1000, 200)):
        est, ed, vd = G.esamp(k, 1, 99, reps=reps, want_draws=True)
        oe, oed, ovd = O.esamp_trial(g.u, g.v, g.nU, g.nV, k, reps, 99, 0)
        assert np.array_equal(u64(ed), oed) and np.array_equal(u64(vd), ovd)
        assert est[0] == pytest.approx(oe, rel=1e-12)
    est, cd, bd = G.wsamp(300, 1, 98, want_draws=True)
    oe, ocd, obd = O.wsamp_trial(g.u, g.v, g.nU, g.nV, 300, 98, 0)
    assert np.array_equal(u64(cd), ocd) and np.array_equal(u64(bd), obd)
    assert est[0] == pytest.approx(oe, rel=1e-12)


def test_vertices_and_edges_of_every_degree_band(big):
    """b_v and b_e of vertices drawn at random from every start-side degree band
    (the kernels' classes split on degree: counter widths at 3, 15 and 255; the
    window classes at 64 and 640 rows; the highest ranks take the hub block or
    the flat expansion), against the oracle computed one by one."""
    g, G = big
    bU, bV, B = G.per_vertex()
    bU = u64(bU)
    be, _ = G.per_edge()
    be = u64(be)
    dU = np.bincount(g.u, minlength=g.nU)
    rng = np.random.default_rng(77)
    ids = []
    for lo, hi in ((2, 3), (4, 15), (16, 64), (65, 255), (256, 640), (641, 1 << 30)):
        pool = np.nonzero((dU >= lo) & (dU <= hi))[0]
        if pool.size:
            ids.append(rng.choice(pool, min(25, pool.size), replace=False))
    ids = np.unique(np.concatenate(ids)).astype(np.uint32)
    assert np.array_equal(bU[ids], O.per_vertex_list(g.u, g.v, g.nU, g.nV, 0, ids))
    # the first and the last edge of each sampled vertex's row (canonical ids)
    offU = np.zeros(g.nU + 1, np.int64)
    np.cumsum(dU, out=offU[1:])
    eidx = np.unique(np.concatenate([offU[ids], offU[ids + 1] - 1])).astype(np.uint64)
    cu, cv = G.edges()
    cu = cu.cpu().numpy().astype(np.uint32)
    cv = cv.cpu().numpy().astype(np.uint32)
    assert np.array_equal(be[eidx.astype(np.int64)], O.per_edge_list(cu, cv, g.nU, g.nV, eidx))
