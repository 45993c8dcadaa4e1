"""Host-side fault injection: a device allocation made to fail at each point of
a call.  Every call returns BFC_ENOMEM cleanly, the handles it was given stay
usable, and once no allocation fails the same call gives the oracle's counts.
No GPU fault is involved: the failure is injected before the allocation."""
import numpy as np
import pytest

import oracle as O
from paper_1801_00338_gb300 import synth

pytestmark = pytest.mark.gpu

ENOMEM = -4


@pytest.fixture(scope="module")
def bfc():
    import torch
    assert torch.cuda.is_available()
    from paper_1801_00338_gb300 import build as B
    B.build()
    from paper_1801_00338_gb300 import bfc as mod
    mod.load()
    yield mod
    mod.bfc_fail_alloc_after(-1)


@pytest.fixture(scope="module")
def medium():
    g = synth.chung_lu_scaled(3000, 9000, 40_000, 2.1, 2.4, 5)
    oB, oside = O.exact(g.u, g.v, g.nU, g.nV)
    return g, oB, oside


def u64(t):
    return t.cpu().numpy().view(np.uint64)


def through_failures(bfc, call, limit=2000):
    """call() with the (n+1)-th device allocation failing, for n = 0, 1, ...,
    until it succeeds; every failed attempt must raise BFC_ENOMEM.  Returns
    (the successful result, the number of failed attempts)."""
    for n in range(limit):
        bfc.bfc_fail_alloc_after(n)
        try:
            out = call()
        except bfc.BfcError as e:
            assert e.code == ENOMEM, e
            continue
        finally:
            bfc.bfc_fail_alloc_after(-1)
        return out, n
    raise AssertionError("the call never succeeded")


def test_graph_build(bfc, medium):
    g, oB, oside = medium
    G, n = through_failures(bfc, lambda: bfc.Graph(g.u, g.v, g.nU, g.nV))
    assert n >= 3
    with G:
        assert G.exact() == (oB, oside)


def test_exact_counts(bfc, medium):
    g, oB, oside = medium
    with bfc.Graph(g.u, g.v, g.nU, g.nV) as G:
        res, n = through_failures(bfc, lambda: G.exact())
        assert res == (oB, oside) and n >= 3
    with bfc.Graph(g.u, g.v, g.nU, g.nV) as G:
        res, n = through_failures(bfc, lambda: G.exact_hub(hubs=128, tau=2))
        assert res[0] == oB and n >= 3
        assert G.exact_hub(hubs=256)[0] == oB


def test_local_counts(bfc, medium):
    g, oB, _ = medium
    oU, oV = O.per_vertex(g.u, g.v, g.nU, g.nV)
    can = O.canonical_ids(g.u, g.v, g.nU, g.nV)
    oe = O.per_edge(g.u, g.v, g.nU, g.nV)
    for whole in (False, True):
        with bfc.Graph(g.u, g.v, g.nU, g.nV) as G:
            (bU, bV, be, B), n = through_failures(bfc, lambda: G.local_counts(whole_rows=whole))
            assert n >= 1
            assert B == oB
            assert np.array_equal(u64(bU), oU) and np.array_equal(u64(bV), oV)
            assert np.array_equal(u64(be)[can], oe)


def test_samplers(bfc, medium):
    g, _, _ = medium
    with bfc.Graph(g.u, g.v, g.nU, g.nV) as G:
        want_v = G.vsamp(200, 3, 11)
        want_e = G.esamp(100, 3, 12)
        want_f = G.esamp(100, 3, 13, reps=10)
        want_w = G.wsamp(100, 3, 14)
    with bfc.Graph(g.u, g.v, g.nU, g.nV) as G:
        got, _ = through_failures(bfc, lambda: G.vsamp(200, 3, 11))
        assert np.array_equal(got, want_v)
        got, _ = through_failures(bfc, lambda: G.esamp(100, 3, 12))
        assert np.array_equal(got, want_e)
        got, _ = through_failures(bfc, lambda: G.esamp(100, 3, 13, reps=10))
        assert np.array_equal(got, want_f)
        got, _ = through_failures(bfc, lambda: G.wsamp(100, 3, 14))
        assert np.array_equal(got, want_w)


def test_batched_exact(bfc):
    params = synth.uneven_batch_params(12, 29, m_lo=100, m_hi=20_000)
    graphs = []
    for i, (nU, nV, m, gamma) in enumerate(params):
        u, v = synth.chung_lu_bipartite(nU, nV, m, gamma, gamma, 700 + i)
        graphs.append((u, v, nU, nV))
    (B, side), n = through_failures(bfc, lambda: bfc.bfc_exact_batch(graphs))
    assert n >= 3
    for (u, v, nU, nV), b, sd in zip(graphs, B, side):
        ob, os_ = O.exact(u, v, nU, nV)
        assert int(b) == ob and int(sd) == os_


ETIMEOUT = -6


def test_hub_wait_gives_up_and_the_handle_recovers(bfc, medium):
    """The hub kernel's bounded waits: with a 1 ns limit the first wait for a
    TMA copy gives up (the copy cannot land that fast), the kernel drains what
    it issued and the call returns BFC_ETIMEOUT; with the limit restored the
    same handle gives the oracle's count, repeatedly."""
    g, oB, _ = medium
    with bfc.Graph(g.u, g.v, g.nU, g.nV) as G:
        try:
            bfc.bfc_set_wait_limit(1)
            with pytest.raises(bfc.BfcError) as ei:
                G.exact_hub(hubs=256, tau=2)
            assert ei.value.code == ETIMEOUT
        finally:
            bfc.bfc_set_wait_limit(0)
        for _ in range(2):
            B, _, st = G.exact_hub(hubs=256, tau=2)
            assert B == oB and st["hubs"] == 256
        assert G.exact()[0] == oB
