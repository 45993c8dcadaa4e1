"""The tensor-core hub block of ExactBFC (bfc_exact_hub / BFC_HUB_MMA) against
the oracle: the count must not depend on the hub set, on the dense-column
threshold tau (all columns dense, all light, or the cost model's choice), or
on the start side.  Counts are integers: every comparison is exact."""
import math

import numpy as np
import pytest

import oracle as O
from paper_1801_00338_gb300 import synth

pytestmark = pytest.mark.gpu

ALL_LIGHT = 1 << 30   # no column reaches it: the int32 pair matrix only
ALL_DENSE = 2         # every column with a hub pair goes to the tensor cores


@pytest.fixture(scope="module")
def bfc():
    import torch
    assert torch.cuda.is_available()
    from paper_1801_00338_gb300 import build as B
    B.build()
    from paper_1801_00338_gb300 import bfc as mod
    mod.load()
    return mod


def test_every_start_vertex_a_hub(bfc):
    """512 start vertices (U forced), all of them hubs: the tile kernel and the
    light-pair matrix count every pair; K spans many 64-wide chunks with a
    ragged last one."""
    u, v = synth.uniform_bipartite(512, 3000, 40_000, 11)
    oB, _ = O.exact(u, v, 512, 3000, side=0)
    with bfc.Graph(u, v, 512, 3000) as G:
        for tau in (ALL_DENSE, 0, 14, ALL_LIGHT):
            B, side, st = G.exact_hub("U", hubs=512, tau=tau)
            assert side == 0 and st["hubs"] == 512
            assert B == oB, (tau, st)
        _, _, st = G.exact_hub("U", hubs=512, tau=ALL_DENSE)
        assert st["K"] > 64 and st["K"] % 64 and st["light_pairs"] == 0
        _, _, st = G.exact_hub("U", hubs=512, tau=ALL_LIGHT)
        assert st["K"] == 0 and st["light_pairs"] > 0


@pytest.mark.parametrize("side", ["U", "V", None])
def test_chung_lu_hub_sizes_and_thresholds(bfc, side):
    g = synth.chung_lu_scaled(3000, 9000, 60_000, 2.1, 2.4, 5)
    oB, _ = O.exact(g.u, g.v, g.nU, g.nV)
    with bfc.Graph(g.u, g.v, g.nU, g.nV) as G:
        assert G.exact(side)[0] == oB
        for hubs in (128, 384, 1024):
            for tau in (ALL_DENSE, 0, 6, ALL_LIGHT):
                B, _, st = G.exact_hub(side, hubs=hubs, tau=tau)
                assert B == oB, (hubs, tau, st)
        B, _ = G.exact(side, hub_mma=True)
        assert B == oB


def test_biclique_closed_form(bfc):
    """K_{384,70}: every pair of U vertices shares all 70 midpoints, so every
    column is dense for any tau <= 384 and c = 70 in every tile entry."""
    a, b = 384, 70
    u, v = synth.complete_bipartite(a, b)
    want = math.comb(a, 2) * math.comb(b, 2)
    with bfc.Graph(u, v, a, b) as G:
        for hubs in (128, 384):
            for tau in (ALL_DENSE, 0, ALL_LIGHT):
                B, side, st = G.exact_hub("U", hubs=hubs, tau=tau)
                assert B == want, (hubs, tau, st)


def test_ragged_start_side_and_automatic_size(bfc):
    """nS = 1000 is not a multiple of 128: the largest hub set is the top 896
    ranks.  The automatic size covers the walk's big class, which this small
    uniform graph does not have (no hubs: the plain walk), as a side smaller
    than 128 never has hubs."""
    u, v = synth.uniform_bipartite(1000, 100, 8000, 4)
    oB, _ = O.exact(u, v, 1000, 100)
    with bfc.Graph(u, v, 1000, 100) as G:
        B, _, st = G.exact_hub("U", hubs=896)
        assert B == oB and st["hubs"] == 896
        for side in ("U", "V"):
            B, _, st = G.exact_hub(side)
            assert B == oB and st["hubs"] == 0
        B, _ = G.exact("U", hub_mma=True)
        assert B == oB


def test_bad_arguments(bfc):
    u, v = synth.uniform_bipartite(300, 200, 3000, 8)
    with bfc.Graph(u, v, 300, 200) as G:
        for hubs, tau in ((100, 0), (384, 0), (128, 1)):
            with pytest.raises(bfc.BfcError):
                G.exact_hub("U", hubs=hubs, tau=tau)
        # the handle still works after the rejected calls
        assert G.exact_hub("U", hubs=256)[0] == O.exact(u, v, 300, 200)[0]


def test_empty_hub_columns(bfc):
    """Hubs with no shared midpoint: no light pairs, no dense columns."""
    # a perfect matching: no butterflies at all
    n = 256
    u = np.arange(n, dtype=np.uint32)
    v = np.arange(n, dtype=np.uint32)
    with bfc.Graph(u, v, n, n) as G:
        B, _, st = G.exact_hub("U", hubs=256)
        assert B == 0 and st["K"] == 0 and st["light_pairs"] == 0
