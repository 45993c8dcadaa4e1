"""The seeded input generators: determinism and the shape promises they make."""
import numpy as np

from paper_1801_00338_gb300 import synth


def test_uniform_graph_is_simple_and_deterministic():
    g1 = synth.uniform_small(1)
    g2 = synth.uniform_small(1)
    assert g1.m == 20000 and (g1.u == g2.u).all() and (g1.v == g2.v).all()
    key = g1.u.astype(np.uint64) * np.uint64(g1.nV) + g1.v
    assert np.unique(key).size == g1.m
    assert g1.u.max() < g1.nU and g1.v.max() < g1.nV


def test_chung_lu_small_is_simple_and_skewed():
    g = synth.chung_lu_scaled(2000, 10000, 50000, 2.1, 2.5, 7)
    key = g.u.astype(np.uint64) * np.uint64(g.nV) + g.v
    assert np.unique(key).size == g.m == 50000
    dU = np.bincount(g.u, minlength=g.nU)
    # a power law: the top 1% of U carries far more than 1% of the edges
    top = np.sort(dU)[::-1][: g.nU // 100].sum()
    assert top > 0.08 * g.m


def test_pareto_weights_hit_the_mean():
    for gamma in (2.0, 2.1, 2.5, 3.0):
        w = synth.pareto_weights(200000, gamma, 15.0, 2e5, 3)
        # heavy tails: the sample mean converges slowly from below
        assert abs(w.mean() / 15.0 - 1) < 0.15


def test_uneven_batch_params():
    ps = synth.uneven_batch_params(200, 5)
    for nU, nV, m, gamma in ps:
        assert 1e3 * 0.99 <= m <= 1e6 * 1.01 and 1.9 <= gamma <= 3.0
        assert nU * nV >= 2 * m


def test_batch_generation_does_not_depend_on_the_worker_count():
    """The batched workload's graphs come out the same whether they are drawn
    in one process or by a pool of spawned workers, and graph i is
    uneven_batch_graph(i, params)."""
    g1 = synth.uneven_batch(12, 5, workers=1, m_hi=2e4)
    g2 = synth.uneven_batch(12, 5, workers=2, m_hi=2e4)
    assert len(g1) == len(g2) == 12
    for a, b in zip(g1, g2):
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1]) and a[2:] == b[2:]
    params = synth.uneven_batch_params(12, 5, m_hi=2e4)
    u, v, nU, nV = synth.uneven_batch_graph(7, params)
    assert np.array_equal(u, g1[7][0]) and (nU, nV) == g1[7][2:]
