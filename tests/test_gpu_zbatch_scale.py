"""The two largest seeded workloads against the oracle's stored counts
(tests/golden/, written by make_full_scale_counts.py from oracle/ alone):
every one of the 4,096 uneven graphs of the batched exact count, and the exact
B of the 300M-edge graph of the sparsification estimators."""
import os

import numpy as np
import pytest

from paper_1801_00338_gb300 import synth

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def bfc():
    import torch
    assert torch.cuda.is_available()
    from paper_1801_00338_gb300 import build as B
    B.build()
    from paper_1801_00338_gb300 import bfc as mod
    mod.load()
    return mod


def _read_batch_golden():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "uneven_batch_4096.txt")) if not ln.startswith("#")]
    a = np.array([[int(x) for x in r] for r in rows], dtype=np.uint64)
    return a[:, 1], a[:, 2], a[:, 3].astype(np.int32)  # m, B, side


def test_all_4096_batched_counts_equal_the_oracle(bfc):
    """One bfc_exact_batch call over the 4,096 graphs (Algorithm 1 per graph,
    start side by its own degree sums): every B and every start side equal the
    oracle's."""
    m, oB, oside = _read_batch_golden()
    assert len(oB) == 4096
    graphs = synth.uneven_batch(4096, 5)
    assert [len(g[0]) for g in graphs] == [int(x) for x in m]
    B, side = bfc.bfc_exact_batch(graphs)
    assert np.array_equal(B.astype(np.uint64), oB)
    assert np.array_equal(side.astype(np.int32), oside)


def test_300m_edge_graph_exact_count_equals_the_oracle(bfc):
    path = os.path.join(GOLDEN, "chung_lu_20m_40m_300m.txt")
    if not os.path.exists(path):
        pytest.skip("stored count not written yet")
    kv = dict(ln.split() for ln in open(path) if not ln.startswith("#"))
    g = synth.chung_lu_scaled(20_000_000, 40_000_000, 300_000_000, 2.0, 2.3, 3)
    assert g.m == int(kv["m"])
    with bfc.Graph(g.u, g.v, g.nU, g.nV) as G:
        del g
        B, side = G.exact()
        assert B == int(kv["B"]) and "UV"[side] == kv["start_side"]
        Bh, _ = G.exact(hub_mma=True)
        assert Bh == B
