"""Pins of the CPU oracle against what the paper and the mathematics fix.

Nothing here calls the CUDA path.  Brute force means listing every butterfly
{a, b} x {x, y} by its definition (Section 2), independently of the oracle's
hash-map counting (Algorithms 1-2).
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_1801_00338_gb300 import synth
from tests.conftest import read_golden


def C2(k):
    return k * (k - 1) // 2


# ----------------------------------------------------------------------------
# published values
# ----------------------------------------------------------------------------

def test_splitmix64_published_outputs(golden_dir):
    for seed, k, want in read_golden(os.path.join(golden_dir, "splitmix64.txt")):
        assert O.splitmix64(seed, k) == want
        assert int(synth.splitmix64(seed, k - 1, 1)[0]) == want


def test_table1_biclique_row(golden_dir):
    """Table 1: the (10^4, 10)-biclique has B = 2,249,775,000 with the printed degree-square sums."""
    (nL, nR, m, sqL, sqR, B), = read_golden(os.path.join(golden_dir, "table1_biclique.txt"))
    u, v = synth.complete_bipartite(nL, nR)
    assert u.size == m
    assert O.degree_square_sums(u, v, nL, nR) == (sqL, sqR)
    got, side = O.exact(u, v, nL, nR)
    assert got == B
    # Algorithm 1, first lines: sum_L d^2 < sum_R d^2, so the start set is R.
    assert side == 1


@pytest.mark.parametrize("a,b", [(2, 2), (2, 7), (5, 3), (9, 9), (1, 6), (13, 4)])
def test_biclique_closed_form(a, b):
    u, v = synth.complete_bipartite(a, b)
    B = C2(a) * C2(b)
    for side in (-1, 0, 1):
        assert O.exact(u, v, a, b, side)[0] == B
    bU, bV = O.per_vertex(u, v, a, b)
    assert (bU == (a - 1) * C2(b)).all()
    assert (bV == (b - 1) * C2(a)).all()
    be = O.per_edge(u, v, a, b)
    assert (be == (a - 1) * (b - 1)).all()


# ----------------------------------------------------------------------------
# brute force on tiny graphs
# ----------------------------------------------------------------------------

def _tiny_graphs(count, seed0):
    rs = synth.uniform01(seed0, 0, 3 * count).reshape(count, 3)
    for i in range(count):
        nU = 1 + int(rs[i, 0] * 10)
        nV = 1 + int(rs[i, 1] * 10)
        m = int(rs[i, 2] * nU * nV)
        if m == 0:
            u = v = np.zeros(0, np.uint32)
        else:
            u, v = synth.uniform_bipartite(nU, nV, m, seed0 + 7919 * i)
        yield nU, nV, u, v


def test_brute_force_500_graphs():
    for nU, nV, u, v in _tiny_graphs(500, 11):
        B, bU, bV, be = O.brute_local(u, v, nU, nV)
        for side in (-1, 0, 1):
            assert O.exact(u, v, nU, nV, side)[0] == B
        oU, oV = O.per_vertex(u, v, nU, nV)
        assert (oU == bU).all() and (oV == bV).all()
        assert (O.per_edge(u, v, nU, nV) == be).all()


def test_dense_random_graphs_vs_brute():
    """Denser graphs (up to 20 x 20) where pair multiplicities reach 10+."""
    for i in range(40):
        nU = 6 + i % 15
        nV = 5 + (3 * i) % 16
        m = int(0.6 * nU * nV)
        u, v = synth.uniform_bipartite(nU, nV, m, 1000 + i)
        B, bU, bV, be = O.brute_local(u, v, nU, nV)
        assert O.exact(u, v, nU, nV)[0] == B
        oU, oV = O.per_vertex(u, v, nU, nV)
        assert (oU == bU).all() and (oV == bV).all()
        assert (O.per_edge(u, v, nU, nV) == be).all()


def test_per_edge_counts_as_a_matrix_product():
    """With A the 0/1 matrix of U rows against V columns and C = A A^T (Lemma 1,
    Eq. (2): C[v, w] = |Gamma_v ^ Gamma_w|), the definition of Section 2 gives
    b_(v,x) = sum over w in Gamma_x, w != v, of (C[v, w] - 1), i.e. the entry
    (v, x) of M A with M = C - 1 off the diagonal and 0 on it.  The oracle's
    per-edge counts must equal it.  The product stays exact when M is split
    into its low and high bytes, each multiplied by A in float32: every operand
    is an integer below 256 (exact in bfloat16 too) and every partial sum of
    one byte product stays below 2^24."""
    for i in range(12):
        nU, nV = 10 + 3 * i, 12 + 2 * i
        m = (nU * nV) // (2 + i % 3)
        u, v = synth.uniform_bipartite(nU, nV, m, 4000 + i)
        A = np.zeros((nU, nV), np.int64)
        A[u, v] = 1
        C = A @ A.T
        M = C - 1
        np.fill_diagonal(M, 0)
        M[C == 0] = 0  # pairs without a common neighbour meet no edge of the sum anyway
        BE = M @ A
        assert np.array_equal(BE[u, v].astype(np.uint64), O.per_edge(u, v, nU, nV))
        lo = (M & 255).astype(np.float32)
        hi = (M >> 8).astype(np.float32)
        Af = A.astype(np.float32)
        split = (hi @ Af).astype(np.int64) * 256 + (lo @ Af).astype(np.int64)
        assert np.array_equal(split, BE)


def test_printed_algorithm3_is_not_b_e():
    """Algorithm 3 as printed (sum of C(C[x], 2) over x in Gamma_v \\ {u}, C[x] counting
    2-paths from u) differs from the definition of b_e; the oracle follows the definition."""
    u, v = synth.uniform_bipartite(8, 8, 40, 5)
    B, _, _, be = O.brute_local(u, v, 8, 8)
    nbrL, nbrR = {}, {}
    for a, x in zip(u.tolist(), v.tolist()):
        nbrL.setdefault(a, set()).add(x)
        nbrR.setdefault(x, set()).add(a)
    printed = []
    for a, x in zip(u.tolist(), v.tolist()):   # e = (u, v) of Algorithm 3 with u := a in L, v := x in R
        Cx = {}
        for w in nbrL[a]:
            for y in nbrR[w]:
                if y in nbrR[x] and y != a:
                    Cx[y] = Cx.get(y, 0) + 1
        printed.append(sum(C2(c) for c in Cx.values()))
    assert list(be) != printed
    assert (O.per_edge(u, v, 8, 8) == be).all()


def test_empty_and_degenerate():
    z = np.zeros(0, np.uint32)
    assert O.exact(z, z, 5, 7)[0] == 0
    bU, bV = O.per_vertex(z, z, 5, 7)
    assert bU.sum() == 0 and bV.sum() == 0
    # a star and a single edge have no butterflies
    u = np.zeros(6, np.uint32); v = np.arange(6, dtype=np.uint32)
    assert O.exact(u, v, 1, 6)[0] == 0
    assert O.exact(u[:1], v[:1], 1, 1)[0] == 0


def test_rejects_bad_input():
    u = np.array([0, 1, 0], np.uint32); v = np.array([0, 1, 0], np.uint32)
    with pytest.raises(RuntimeError):
        O.exact(u, v, 2, 2)          # duplicate edge
    with pytest.raises(RuntimeError):
        O.exact(np.array([5], np.uint32), np.array([0], np.uint32), 2, 2)  # id out of range


# ----------------------------------------------------------------------------
# invariants on a mid-size graph
# ----------------------------------------------------------------------------

@pytest.fixture(scope="module")
def uniform_small():
    return synth.uniform_small()


def test_lemma1_identities(uniform_small):
    g = uniform_small
    B, side = O.exact(g.u, g.v, g.nU, g.nV)
    assert B > 0
    assert O.exact(g.u, g.v, g.nU, g.nV, 0)[0] == B
    assert O.exact(g.u, g.v, g.nU, g.nV, 1)[0] == B
    bU, bV = O.per_vertex(g.u, g.v, g.nU, g.nV)
    # Eq. (1): each butterfly has two vertices on each side
    assert int(bU.sum()) == 2 * B and int(bV.sum()) == 2 * B
    be = O.per_edge(g.u, g.v, g.nU, g.nV)
    # each butterfly has four edges
    assert int(be.sum()) == 4 * B
    # b_x = 1/2 sum of b_e over the edges at x (each butterfly through x uses two of its edges)
    sU = np.zeros(g.nU, np.uint64); np.add.at(sU, g.u, be)
    sV = np.zeros(g.nV, np.uint64); np.add.at(sV, g.v, be)
    assert (sU == 2 * bU).all() and (sV == 2 * bV).all()


def test_relabel_invariance(uniform_small):
    g = uniform_small
    B, _ = O.exact(g.u, g.v, g.nU, g.nV)
    pu = np.argsort(synth.splitmix64(77, 0, g.nU)).astype(np.uint32)
    pv = np.argsort(synth.splitmix64(78, 0, g.nV)).astype(np.uint32)
    u2, v2 = pu[g.u], pv[g.v]
    assert O.exact(u2, v2, g.nU, g.nV)[0] == B
    # swapping the sides gives the same count
    assert O.exact(g.v, g.u, g.nV, g.nU)[0] == B
    bU, bV = O.per_vertex(g.u, g.v, g.nU, g.nV)
    cU, cV = O.per_vertex(u2, v2, g.nU, g.nV)
    assert (cU[pu] == bU).all() and (cV[pv] == bV).all()


def test_lists_match_full_arrays(uniform_small):
    g = uniform_small
    bU, bV = O.per_vertex(g.u, g.v, g.nU, g.nV)
    ids = np.arange(0, g.nU, 37, dtype=np.uint32)
    assert (O.per_vertex_list(g.u, g.v, g.nU, g.nV, 0, ids) == bU[ids]).all()
    ids = np.arange(0, g.nV, 41, dtype=np.uint32)
    assert (O.per_vertex_list(g.u, g.v, g.nU, g.nV, 1, ids) == bV[ids]).all()
    be = O.per_edge(g.u, g.v, g.nU, g.nV)
    idx = np.arange(0, g.m, 97, dtype=np.uint64)
    assert (O.per_edge_list(g.u, g.v, g.nU, g.nV, idx) == be[idx]).all()


def test_canonical_ids_are_lexicographic_ranks(uniform_small):
    g = uniform_small
    can = O.canonical_ids(g.u, g.v, g.nU, g.nV)
    key = g.u.astype(np.uint64) * np.uint64(g.nV) + g.v.astype(np.uint64)
    assert (np.argsort(key) == np.argsort(can)).all()
    assert sorted(can.tolist()) == list(range(g.m))


def test_prepared_partial_sums(uniform_small):
    g = uniform_small
    B, side = O.exact(g.u, g.v, g.nU, g.nV)
    n = g.nU if side == 0 else g.nV
    P = O.Prepared(g.u, g.v, g.nU, g.nV, side)
    s, paths = P.count(np.arange(n, dtype=np.uint32))
    assert s == 2 * B
    mid = np.bincount(g.v if side == 0 else g.u, minlength=g.nV if side == 0 else g.nU).astype(np.int64)
    # every 2-path v -> u -> w (w != v) with u on the other side, walked from both ends: 2 * sum C(d_u, 2)
    assert paths == int((mid * (mid - 1)).sum())


# ----------------------------------------------------------------------------
# sparsification estimators
# ----------------------------------------------------------------------------

def _kept_by_hash(g, p, seed, t):
    """ESpar keep mask over canonical ids, computed here from the generator's own SplitMix64."""
    T = int(p * 4294967296.0)
    ts = int(synth.splitmix64(seed, t, 1)[0])
    h = synth.splitmix64(ts, 0, g.m) >> np.uint64(32)
    return h < np.uint64(T), T


def test_espar_trial_equals_count_of_kept_edges():
    g = synth.Graph(*synth.uniform_bipartite(12, 14, 90, 3), 12, 14)
    can = O.canonical_ids(g.u, g.v, g.nU, g.nV)
    for t in range(6):
        keep_c, T = _kept_by_hash(g, 0.6, 99, t)
        keep = keep_c[can]
        want = len(O.butterflies(g.u[keep], g.v[keep]))
        beta, est = O.espar_trial(g.u, g.v, g.nU, g.nV, 0.6, 99, t)
        assert beta == want
        s = 4294967296.0 / T
        assert est == beta * ((s * s) * (s * s))


def test_clrspar_trial_equals_count_of_monochromatic_edges():
    g = synth.Graph(*synth.uniform_bipartite(12, 14, 90, 4), 12, 14)
    N = 3
    for t in range(6):
        ts = int(synth.splitmix64(5, t, 1)[0])
        r = synth.splitmix64(ts, 0, g.nU + g.nV) >> np.uint64(32)
        col = ((r * np.uint64(N)) >> np.uint64(32)).astype(np.int64)
        keep = col[g.u] == col[g.nU + g.v.astype(np.int64)]
        want = len(O.butterflies(g.u[keep], g.v[keep]))
        beta, est = O.clrspar_trial(g.u, g.v, g.nU, g.nV, N, 5, t)
        assert beta == want and est == beta * 27.0


def _small_with_pairs(seed, nU=4, nV=5, m=13):
    u, v = synth.uniform_bipartite(nU, nV, m, seed)
    return u, v, nU, nV


def test_espar_moments_by_enumeration():
    """E[Y] = B and Var[Y] from Lemma 8, checked over all 2^m edge subsets."""
    for seed in (1, 2, 3):
        u, v, nU, nV = _small_with_pairs(seed)
        B, _ = O.exact(u, v, nU, nV)
        pairs = O.pair_types(u, v)
        assert sum(pairs.values()) == C2(B)
        m = u.size
        for p in (0.2, 0.5):
            E = E2 = 0.0
            for mask in range(1 << m):
                sel = [i for i in range(m) if mask >> i & 1]
                pr = p ** len(sel) * (1 - p) ** (m - len(sel))
                y = len(O.butterflies(u[sel], v[sel])) / p ** 4 if sel else 0.0
                E += pr * y
                E2 += pr * y * y
            assert E == pytest.approx(B, rel=1e-9)
            assert E2 - E * E == pytest.approx(O.espar_variance(B, pairs, p), rel=1e-9)


def test_clrspar_moments_by_enumeration():
    """E[Y] = B and Var[Y] from Lemma 9, checked over all N^n colourings."""
    import itertools
    for seed, N in ((4, 2), (5, 3)):
        u, v, nU, nV = _small_with_pairs(seed, 3, 4, 9)
        B, _ = O.exact(u, v, nU, nV)
        pairs = O.pair_types(u, v)
        n = nU + nV
        E = E2 = 0.0
        w = 1.0 / N ** n
        for col in itertools.product(range(N), repeat=n):
            keep = np.array([col[a] == col[nU + x] for a, x in zip(u.tolist(), v.tolist())])
            y = len(O.butterflies(u[keep], v[keep])) * N ** 3 if keep.any() else 0
            E += w * y
            E2 += w * y * y
        assert E == pytest.approx(B, rel=1e-9)
        assert E2 - E * E == pytest.approx(O.clrspar_variance(B, pairs, N), rel=1e-9)


def test_espar_mean_of_1000_trials_within_3_se():
    u, v = synth.uniform_bipartite(10, 10, 45, 8)
    B, _ = O.exact(u, v, 10, 10)
    pairs = O.pair_types(u, v)
    p = 0.5
    T = O.espar_threshold(p)
    ests = [O.espar_trial(u, v, 10, 10, p, 2024, t)[1] for t in range(1000)]
    var = O.espar_variance(B, pairs, T / 4294967296.0)
    assert abs(np.mean(ests) - B) <= 3 * math.sqrt(var / 1000)


# ----------------------------------------------------------------------------
# vertex sampling
# ----------------------------------------------------------------------------

def test_vsamp_uniform_draws_and_estimate():
    g = synth.Graph(*synth.uniform_bipartite(15, 12, 80, 9), 15, 12)
    bU, bV = O.per_vertex(g.u, g.v, g.nU, g.nV)
    b = np.concatenate([bU, bV]).astype(np.float64)
    n = g.nU + g.nV
    k = 25
    est, drawn, bd = O.vsamp_trial(g.u, g.v, g.nU, g.nV, k, 31, 2)
    ts = int(synth.splitmix64(31, 2, 1)[0])
    r = synth.splitmix64(ts, 0, 2 * k).reshape(k, 2)[:, 1]
    want_idx = [(int(x) * n) >> 64 for x in r]
    assert drawn.tolist() == want_idx
    assert (bd == b[want_idx]).all()
    assert est == pytest.approx(np.mean(b[want_idx] * n / 4.0), rel=1e-12)
    # Lemma 4: the single-draw estimator is unbiased, sum_v (1/n) (b_v n / 4) = B
    B, _ = O.exact(g.u, g.v, g.nU, g.nV)
    assert np.sum(b * n / 4.0) / n == pytest.approx(B, rel=1e-12)


def test_vsamp_weighted_is_unbiased_and_follows_prefix_rule():
    g = synth.Graph(*synth.uniform_bipartite(15, 12, 80, 10), 15, 12)
    n = g.nU + g.nV
    w = (synth.splitmix64(3, 0, n) >> np.uint64(40)).astype(np.uint32) + 1
    bU, bV = O.per_vertex(g.u, g.v, g.nU, g.nV)
    b = np.concatenate([bU, bV]).astype(np.float64)
    B, _ = O.exact(g.u, g.v, g.nU, g.nV)
    q = O.mixture_q(w)
    assert np.sum(q * b / (4 * q)) == pytest.approx(B, rel=1e-12)
    k = 40
    est, drawn, bd = O.vsamp_trial(g.u, g.v, g.nU, g.nV, k, 7, 0, weights=w)
    ts = int(synth.splitmix64(7, 0, 1)[0])
    r = synth.splitmix64(ts, 0, 2 * k).reshape(k, 2)
    pref = np.cumsum(w.astype(np.uint64))
    W = int(pref[-1])
    want = []
    for r1, r2 in r.tolist():
        if r1 >> 63 == 0:
            want.append((r2 * n) >> 64)
        else:
            want.append(int(np.searchsorted(pref, (r2 * W) >> 64, side="right")))
    assert drawn.tolist() == want
    assert est == pytest.approx(np.mean(b[want] / (4 * q[want])), rel=1e-12)


def test_vsamp_mean_of_trials_within_3_se():
    g = synth.Graph(*synth.uniform_bipartite(20, 20, 150, 12), 20, 20)
    bU, bV = O.per_vertex(g.u, g.v, g.nU, g.nV)
    b = np.concatenate([bU, bV])
    B, _ = O.exact(g.u, g.v, g.nU, g.nV)
    k = 10
    ests = [O.vsamp_trial(g.u, g.v, g.nU, g.nV, k, 5, t)[0] for t in range(1000)]
    var = O.vsamp_variance(b) / k
    assert abs(np.mean(ests) - B) <= 3 * math.sqrt(var / 1000)
    # the sample variance of the trials agrees with the exact one
    assert np.var(ests) == pytest.approx(var, rel=0.15)


# ----------------------------------------------------------------------------
# edge sampling (Algorithm 5) and the fast per-edge estimate (Algorithm 7)
# ----------------------------------------------------------------------------

def _dense(nU, nV, p, seed):
    r = synth.uniform01(seed, 0, nU * nV).reshape(nU, nV)
    a, x = np.nonzero(r < p)
    return a.astype(np.uint32), x.astype(np.uint32)


def _adj(u, v, nU, nV):
    rows = [sorted(v[u == a].tolist()) for a in range(nU)]
    cols = [sorted(u[v == x].tolist()) for x in range(nV)]
    return rows, cols


def test_esamp_second_moment_matches_pair_types():
    """Var of Algorithm 5's term is (m/16) sum_e b_e^2 - B^2, and
    sum_e b_e^2 = 4B + 2 p_1e + 4 p_1w (ordered pairs of distinct butterflies
    sharing one edge or two): b_e from the definition against the brute-force
    pair classification; the paper's bound Var <= (m/4)(B + p_E) holds."""
    for seed in (1, 2, 3):
        u, v = _dense(7, 8, 0.55, seed)
        B, _ = O.exact(u, v, 7, 8)
        be = O.per_edge(u, v, 7, 8).astype(np.float64)
        pairs = O.pair_types(u, v)
        assert len(O.butterflies(u, v)) == B
        assert be.sum() == 4 * B
        assert int((be * be).sum()) == 4 * B + 2 * pairs["1e"] + 4 * pairs["1w"]
        m = u.size
        var = O.esamp_term_variance(be, None, None, 0)
        assert var == pytest.approx(m / 16.0 * (4 * B + 2 * pairs["1e"] + 4 * pairs["1w"]) - B * B, rel=1e-12)
        assert var <= m / 4.0 * (B + pairs["1e"] + pairs["1w"])


def test_fast_ebfc_expectation_by_enumeration():
    """Algorithm 7 on edge (a, x): over all d_x * d_a equally likely choices of
    a2 in Gamma_x and x2 in Gamma_a (full lists, a2 = a or x2 = x a miss), the
    hits are exactly the butterflies through the edge, so E[Y] = b_e; one
    repetition has variance b_e d_a d_x - b_e^2 <= b_e d_a d_x."""
    u, v = _dense(8, 7, 0.5, 4)
    rows, cols = _adj(u, v, 8, 7)
    E = set(zip(u.tolist(), v.tolist()))
    be = O.per_edge(u, v, 8, 7)
    bf = O.butterflies(u, v)
    for i, (a, x) in enumerate(zip(u.tolist(), v.tolist())):
        hits = sum(1 for a2 in cols[x] for x2 in rows[a] if a2 != a and x2 != x and (a2, x2) in E)
        assert hits == be[i]
        assert hits == sum(1 for (p, q, y, z) in bf if a in (p, q) and x in (y, z))
        dd = len(rows[a]) * len(cols[x])
        mean = hits / dd * dd
        second = hits / dd * dd * dd
        assert second - mean * mean == pytest.approx(be[i] * dd - be[i] ** 2)


def test_esamp_draws_recomputed():
    """The oracle's draw rule recomputed with Python integers: the edge of draw
    j, and for Algorithm 7 the two neighbour picks of every repetition."""
    nU, nV = 9, 10
    u, v = _dense(nU, nV, 0.5, 5)
    m = u.size
    order = np.lexsort((v, u))
    cu, cv = u[order].tolist(), v[order].tolist()   # canonical order
    rows, cols = _adj(u, v, nU, nV)
    E = set(zip(cu, cv))
    be = O.per_edge(u, v, nU, nV)[order]
    k, reps, seed, t = 12, 7, 77, 3
    ts = int(synth.splitmix64(seed, t, 1)[0])
    for r in (0, reps):
        est, edges, vals = O.esamp_trial(u, v, nU, nV, k, r, seed, t)
        terms = []
        for j in range(k):
            ds = int(synth.splitmix64(ts, j, 1)[0])
            out = [int(z) for z in synth.splitmix64(ds, 0, 2 * r + 3)]
            e = (out[0] * m) >> 64
            assert int(edges[j]) == e
            a, x = cu[e], cv[e]
            if r == 0:
                assert int(vals[j]) == be[e]
                terms.append(be[e] * m / 4.0)
            else:
                da, dx = len(rows[a]), len(cols[x])
                h = 0
                for i in range(r):
                    a2 = cols[x][(out[2 * i + 1] * dx) >> 64]
                    x2 = rows[a][(out[2 * i + 2] * da) >> 64]
                    h += a2 != a and x2 != x and (a2, x2) in E
                assert int(vals[j]) == h
                terms.append(h * da * dx / r * m / 4.0)
        assert est == pytest.approx(np.mean(terms), rel=1e-12)


@pytest.mark.parametrize("reps", [0, 10])
def test_esamp_mean_of_trials_within_3_se(reps):
    nU, nV = 12, 14
    u, v = _dense(nU, nV, 0.45, 6)
    B, _ = O.exact(u, v, nU, nV)
    be = O.per_edge(u, v, nU, nV)
    dA = np.bincount(u, minlength=nU)[u]
    dX = np.bincount(v, minlength=nV)[v]
    k, T = 5, 1000
    ests = [O.esamp_trial(u, v, nU, nV, k, reps, 11, t)[0] for t in range(T)]
    var = O.esamp_term_variance(be, dA, dX, reps) / k
    assert abs(np.mean(ests) - B) <= 3 * math.sqrt(var / T)
    assert np.var(ests) == pytest.approx(var, rel=0.15)


# ----------------------------------------------------------------------------
# wedge sampling (Algorithm 6)
# ----------------------------------------------------------------------------

def test_wsamp_moments_by_wedge_enumeration():
    """Over all h wedges (both sides as centres): sum beta = 4B (each butterfly
    has four wedges) and sum beta^2 = 4B + 2 p_1w (ordered pairs sharing a
    wedge), so Var of one term (h/16) sum beta^2 - B^2 stays within the
    paper's bound (h/4)(B + p_1w)."""
    for seed in (7, 8):
        u, v = _dense(7, 9, 0.5, seed)
        B, _ = O.exact(u, v, 7, 9)
        W = O.wedges(u, v, 7, 9)
        dU = np.bincount(u, minlength=7)
        dV = np.bincount(v, minlength=9)
        h = int((dU * (dU - 1) // 2).sum() + (dV * (dV - 1) // 2).sum())
        assert len(W) == h
        beta = np.array([w[3] for w in W], np.int64)
        pairs = O.pair_types(u, v)
        assert beta.sum() == 4 * B
        assert int((beta * beta).sum()) == 4 * B + 2 * pairs["1w"]
        var = h / 16.0 * (beta * beta).sum() - B * B
        assert var <= h / 4.0 * (B + pairs["1w"])


def test_wsamp_draws_recomputed():
    nU, nV = 8, 11
    u, v = _dense(nU, nV, 0.45, 9)
    rows, cols = _adj(u, v, nU, nV)
    adj = rows + cols
    d = np.array([len(r) for r in adj], np.int64)
    c2 = d * (d - 1) // 2
    pref = np.cumsum(c2)
    h = int(pref[-1])
    k, seed, t = 30, 5, 2
    est, cen, beta = O.wsamp_trial(u, v, nU, nV, k, seed, t)
    ts = int(synth.splitmix64(seed, t, 1)[0])
    terms = []
    for j in range(k):
        ds = int(synth.splitmix64(ts, j, 1)[0])
        r1, r2, r3 = (int(z) for z in synth.splitmix64(ds, 0, 3))
        c = int(np.searchsorted(pref, (r1 * h) >> 64, side="right"))
        p = (r2 * int(d[c])) >> 64
        q = (r3 * (int(d[c]) - 1)) >> 64
        q += q >= p
        a, b = adj[c][p], adj[c][q]
        other = cols if c < nU else rows
        bt = len(set(other[a]) & set(other[b])) - 1
        assert int(cen[j]) == c and int(beta[j]) == bt
        terms.append(bt * h / 4.0)
    assert est == pytest.approx(np.mean(terms), rel=1e-12)


def test_wsamp_mean_of_trials_within_3_se():
    nU, nV = 12, 13
    u, v = _dense(nU, nV, 0.4, 10)
    B, _ = O.exact(u, v, nU, nV)
    W = O.wedges(u, v, nU, nV)
    h = len(W)
    beta = np.array([w[3] for w in W], np.float64)
    var1 = h / 16.0 * (beta * beta).sum() - B * B
    k, T = 5, 1000
    ests = [O.wsamp_trial(u, v, nU, nV, k, 21, t)[0] for t in range(T)]
    assert abs(np.mean(ests) - B) <= 3 * math.sqrt(var1 / k / T)
    assert np.var(ests) == pytest.approx(var1 / k, rel=0.15)
