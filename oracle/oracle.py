"""Python face of the butterfly-counting oracle (test infrastructure only).

Only the tests, the smoke check and the benchmark's CPU-baseline leg use this
module.  It wraps the plain C oracle in ``bfc_oracle.c`` (compiled with gcc by
:func:`build`) and adds the closed forms the paper gives for the estimators'
moments.  Nothing here is shared with the CUDA path.

Paper references (arXiv 1801.00338):
  * Lemma 1, Eq. (1)-(3): B, b_v; Algorithm 1: ExactBFC; Algorithm 2: vBFC
  * Section 2: butterfly, b_e definitions; Algorithm 3: eBFC (see bfc_oracle.c)
  * Algorithm 4 / Lemma 4: VSamp; Algorithm 8 / Lemma 8: ESpar;
    Algorithm 9 / Lemma 9: ClrSpar; Section 5: butterfly pair types
  * Algorithm 5: ESamp (exact b_e per draw); Algorithm 7: the fast per-edge
    estimate used in its place; Algorithm 6: WSamp (Section 5.3 for the
    prefix-sum centre draw)
"""
from __future__ import annotations

import ctypes
import itertools
import os
import subprocess
from collections import defaultdict

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bfc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc into oracle/liboracle.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-Wall", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        u32, u64, i32, dbl = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_double
        P = ctypes.c_void_p
        L.orc_degree_square_sums.argtypes = [u32, u32, u64, P, P, P]
        L.orc_exact.argtypes = [u32, u32, u64, P, P, i32, P, P]
        L.orc_per_vertex.argtypes = [u32, u32, u64, P, P, P, P]
        L.orc_per_vertex_list.argtypes = [u32, u32, u64, P, P, i32, u64, P, P]
        L.orc_per_edge.argtypes = [u32, u32, u64, P, P, P]
        L.orc_per_edge_list.argtypes = [u32, u32, u64, P, P, u64, P, P]
        L.orc_canonical_ids.argtypes = [u32, u32, u64, P, P, P]
        L.orc_splitmix64.argtypes = [u64, u64]
        L.orc_splitmix64.restype = u64
        L.orc_espar_trial.argtypes = [u32, u32, u64, P, P, u32, u64, u32, P, P]
        L.orc_clrspar_trial.argtypes = [u32, u32, u64, P, P, u32, u64, u32, P, P]
        L.orc_vsamp_trial.argtypes = [u32, u32, u64, P, P, u64, P, u64, u32, P, P, P]
        L.orc_esamp_trial.argtypes = [u32, u32, u64, P, P, u64, u32, u64, u32, P, P, P]
        L.orc_wsamp_trial.argtypes = [u32, u32, u64, P, P, u64, u64, u32, P, P, P]
        L.orc_prepare.argtypes = [u32, u32, u64, P, P, i32]
        L.orc_prepare.restype = P
        L.orc_prepared_count.argtypes = [P, u64, P, P, P]
        L.orc_prepared_free.argtypes = [P]
        for f in ("orc_degree_square_sums", "orc_exact", "orc_per_vertex", "orc_per_vertex_list",
                  "orc_per_edge", "orc_per_edge_list", "orc_canonical_ids", "orc_espar_trial",
                  "orc_clrspar_trial", "orc_vsamp_trial", "orc_esamp_trial", "orc_wsamp_trial",
                  "orc_prepared_count"):
            getattr(L, f).restype = i32
        _lib = L
    return _lib


def _arr(a, dt):
    a = np.ascontiguousarray(a, dtype=dt)
    return a, a.ctypes.data


def _check(rc: int, what: str):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def _edges(u, v):
    u, pu = _arr(u, np.uint32)
    v, pv = _arr(v, np.uint32)
    if u.size != v.size:
        raise ValueError("u and v differ in length")
    return u, v, pu, pv


# ----------------------------------------------------------------------------
# exact counts
# ----------------------------------------------------------------------------

def degree_square_sums(u, v, nU, nV):
    """(sum_{L} d^2, sum_{R} d^2), the Table 1 columns."""
    u, v, pu, pv = _edges(u, v)
    out = np.zeros(2, np.uint64)
    _check(lib().orc_degree_square_sums(nU, nV, u.size, pu, pv, out.ctypes.data), "degree sums")
    return int(out[0]), int(out[1])


def exact(u, v, nU, nV, side: int = -1):
    """ExactBFC (Algorithm 1).  side -1: the paper's choice, 0: start from L, 1: from R.

    Returns (B, start side used)."""
    u, v, pu, pv = _edges(u, v)
    B = np.zeros(1, np.uint64)
    s = np.zeros(1, np.int32)
    _check(lib().orc_exact(nU, nV, u.size, pu, pv, side, B.ctypes.data, s.ctypes.data), "exact")
    return int(B[0]), int(s[0])


def per_vertex(u, v, nU, nV):
    """vBFC (Algorithm 2) for every vertex: (b over L, b over R), uint64 arrays."""
    u, v, pu, pv = _edges(u, v)
    bU = np.zeros(nU, np.uint64)
    bV = np.zeros(nV, np.uint64)
    _check(lib().orc_per_vertex(nU, nV, u.size, pu, pv, bU.ctypes.data, bV.ctypes.data), "per_vertex")
    return bU, bV


def per_vertex_list(u, v, nU, nV, side: int, ids):
    u, v, pu, pv = _edges(u, v)
    ids, pids = _arr(ids, np.uint32)
    out = np.zeros(ids.size, np.uint64)
    _check(lib().orc_per_vertex_list(nU, nV, u.size, pu, pv, side, ids.size, pids, out.ctypes.data),
           "per_vertex_list")
    return out


def per_edge(u, v, nU, nV):
    """b_e of every edge, in INPUT order."""
    u, v, pu, pv = _edges(u, v)
    out = np.zeros(u.size, np.uint64)
    _check(lib().orc_per_edge(nU, nV, u.size, pu, pv, out.ctypes.data), "per_edge")
    return out


def per_edge_list(u, v, nU, nV, idx):
    u, v, pu, pv = _edges(u, v)
    idx, pidx = _arr(idx, np.uint64)
    out = np.zeros(idx.size, np.uint64)
    _check(lib().orc_per_edge_list(nU, nV, u.size, pu, pv, idx.size, pidx, out.ctypes.data), "per_edge_list")
    return out


def canonical_ids(u, v, nU, nV):
    u, v, pu, pv = _edges(u, v)
    out = np.zeros(u.size, np.uint64)
    _check(lib().orc_canonical_ids(nU, nV, u.size, pu, pv, out.ctypes.data), "canonical_ids")
    return out


def splitmix64(seed: int, k: int) -> int:
    return int(lib().orc_splitmix64(seed & 0xFFFFFFFFFFFFFFFF, k))


# ----------------------------------------------------------------------------
# estimators, one trial at a time
# ----------------------------------------------------------------------------

def espar_threshold(p: float) -> int:
    """The keep threshold T = floor(p * 2^32): an edge is kept iff its 32-bit hash < T."""
    T = int(p * 4294967296.0)
    if not 0 < T <= 0xFFFFFFFF:
        raise ValueError("p out of range")
    return T


def espar_trial(u, v, nU, nV, p: float, seed: int, t: int):
    """One ESpar trial (Algorithm 8): (beta, beta * p^-4) with p = T / 2^32."""
    u, v, pu, pv = _edges(u, v)
    beta = np.zeros(1, np.uint64)
    est = np.zeros(1, np.float64)
    _check(lib().orc_espar_trial(nU, nV, u.size, pu, pv, espar_threshold(p), seed & 0xFFFFFFFFFFFFFFFF, t,
                                 beta.ctypes.data, est.ctypes.data), "espar")
    return int(beta[0]), float(est[0])


def clrspar_trial(u, v, nU, nV, N: int, seed: int, t: int):
    """One ClrSpar trial (Algorithm 9): (beta, beta * N^3)."""
    u, v, pu, pv = _edges(u, v)
    beta = np.zeros(1, np.uint64)
    est = np.zeros(1, np.float64)
    _check(lib().orc_clrspar_trial(nU, nV, u.size, pu, pv, N, seed & 0xFFFFFFFFFFFFFFFF, t,
                                   beta.ctypes.data, est.ctypes.data), "clrspar")
    return int(beta[0]), float(est[0])


def vsamp_trial(u, v, nU, nV, k: int, seed: int, t: int, weights=None):
    """One VSamp trial of k draws (Algorithm 4, or its weighted mixture form).

    Returns (estimate, drawn population indices, b of each draw)."""
    u, v, pu, pv = _edges(u, v)
    pw = None
    if weights is not None:
        weights, pw = _arr(weights, np.uint32)
        if weights.size != nU + nV:
            raise ValueError("weights must cover L then R")
    est = np.zeros(1, np.float64)
    drawn = np.zeros(max(k, 1), np.uint64)
    bd = np.zeros(max(k, 1), np.uint64)
    _check(lib().orc_vsamp_trial(nU, nV, u.size, pu, pv, k, pw, seed & 0xFFFFFFFFFFFFFFFF, t,
                                 est.ctypes.data, drawn.ctypes.data, bd.ctypes.data), "vsamp")
    return float(est[0]), drawn[:k], bd[:k]


def esamp_trial(u, v, nU, nV, k: int, reps: int, seed: int, t: int):
    """One ESamp trial of k edge draws (Algorithm 5).  reps = 0: exact b_e per
    draw; reps > 0: Algorithm 7 repeated reps times per draw.

    Returns (estimate, canonical edge ids drawn, value of each draw: b_e or
    the hit count)."""
    u, v, pu, pv = _edges(u, v)
    est = np.zeros(1, np.float64)
    edges = np.zeros(max(k, 1), np.uint64)
    vals = np.zeros(max(k, 1), np.uint64)
    _check(lib().orc_esamp_trial(nU, nV, u.size, pu, pv, k, reps, seed & 0xFFFFFFFFFFFFFFFF, t,
                                 est.ctypes.data, edges.ctypes.data, vals.ctypes.data), "esamp")
    return float(est[0]), edges[:k], vals[:k]


def wsamp_trial(u, v, nU, nV, k: int, seed: int, t: int):
    """One WSamp trial of k wedge draws (Algorithm 6).

    Returns (estimate, population index of each centre, beta of each draw)."""
    u, v, pu, pv = _edges(u, v)
    est = np.zeros(1, np.float64)
    cen = np.zeros(max(k, 1), np.uint64)
    beta = np.zeros(max(k, 1), np.uint64)
    _check(lib().orc_wsamp_trial(nU, nV, u.size, pu, pv, k, seed & 0xFFFFFFFFFFFFFFFF, t,
                                 est.ctypes.data, cen.ctypes.data, beta.ctypes.data), "wsamp")
    return float(est[0]), cen[:k], beta[:k]


class Prepared:
    """A graph prepared once, for timing Algorithm 1's per-start-vertex loops."""

    def __init__(self, u, v, nU, nV, side: int):
        u, v, pu, pv = _edges(u, v)
        self._h = lib().orc_prepare(nU, nV, u.size, pu, pv, side)
        if not self._h:
            raise RuntimeError("oracle prepare failed")

    def count(self, ids):
        ids, pids = _arr(ids, np.uint32)
        s = np.zeros(1, np.uint64)
        w = np.zeros(1, np.uint64)
        _check(lib().orc_prepared_count(self._h, ids.size, pids, s.ctypes.data, w.ctypes.data), "prepared")
        return int(s[0]), int(w[0])

    def close(self):
        if self._h:
            lib().orc_prepared_free(self._h)
            self._h = None

    def __del__(self):
        self.close()


# ----------------------------------------------------------------------------
# brute force over 4-sets (Section 2 definitions), for tiny graphs
# ----------------------------------------------------------------------------

def butterflies(u, v):
    """Every butterfly {a, b} x {x, y} with all four edges present, as tuples (a, b, x, y), a < b, x < y."""
    nbr = defaultdict(set)
    for a, x in zip(np.asarray(u).tolist(), np.asarray(v).tolist()):
        nbr[a].add(x)
    Ls = sorted(nbr)
    out = []
    for a, b in itertools.combinations(Ls, 2):
        common = sorted(nbr[a] & nbr[b])
        for x, y in itertools.combinations(common, 2):
            out.append((a, b, x, y))
    return out


def brute_local(u, v, nU, nV):
    """(B, b over L, b over R, b_e in input order) by listing every butterfly."""
    bf = butterflies(u, v)
    bU = np.zeros(nU, np.int64)
    bV = np.zeros(nV, np.int64)
    eid = {(a, x): i for i, (a, x) in enumerate(zip(np.asarray(u).tolist(), np.asarray(v).tolist()))}
    be = np.zeros(len(eid), np.int64)
    for a, b, x, y in bf:
        bU[a] += 1; bU[b] += 1; bV[x] += 1; bV[y] += 1
        for e in ((a, x), (a, y), (b, x), (b, y)):
            be[eid[e]] += 1
    return len(bf), bU, bV, be


def pair_types(u, v):
    """Counts of unordered pairs of distinct butterflies by type (Section 5):
    0v (no common vertex), 1v (one), 2v (two, no common edge), 1e (one common
    edge), 1w (a common wedge: three vertices, two edges)."""
    bf = butterflies(u, v)
    verts = [frozenset([("L", a), ("L", b), ("R", x), ("R", y)]) for a, b, x, y in bf]
    edges = [frozenset([(a, x), (a, y), (b, x), (b, y)]) for a, b, x, y in bf]
    cnt = {"0v": 0, "1v": 0, "2v": 0, "1e": 0, "1w": 0}
    for i in range(len(bf)):
        for j in range(i + 1, len(bf)):
            sv = len(verts[i] & verts[j])
            se = len(edges[i] & edges[j])
            if sv == 0:
                cnt["0v"] += 1
            elif sv == 1:
                cnt["1v"] += 1
            elif sv == 2 and se == 0:
                cnt["2v"] += 1
            elif sv == 2 and se == 1:
                cnt["1e"] += 1
            elif sv == 3 and se == 2:
                cnt["1w"] += 1
            else:
                raise AssertionError("pair of butterflies outside the five types")
    return cnt


# ----------------------------------------------------------------------------
# exact moments of the estimators
# ----------------------------------------------------------------------------

def espar_variance(B: int, pairs: dict, p: float) -> float:
    """Var[beta * p^-4] of ESpar (Lemma 8's first line), with the pair counts
    taken over unordered pairs, so that each enters the covariance sum twice:
    p^-8 [B (p^4 - p^8) + 2 p_1e (p^7 - p^8) + 2 p_1w (p^6 - p^8)]."""
    return p ** -8 * (B * (p ** 4 - p ** 8) + 2 * pairs["1e"] * (p ** 7 - p ** 8)
                      + 2 * pairs["1w"] * (p ** 6 - p ** 8))


def clrspar_variance(B: int, pairs: dict, N: int) -> float:
    """Var[beta * N^3] of ClrSpar (Lemma 9's first line), unordered pair counts
    entering twice: p^-6 [B (p^3 - p^6) + 2 (p_2v + p_1e)(p^5 - p^6) + 2 p_1w (p^4 - p^6)], p = 1/N."""
    p = 1.0 / N
    return p ** -6 * (B * (p ** 3 - p ** 6) + 2 * (pairs["2v"] + pairs["1e"]) * (p ** 5 - p ** 6)
                      + 2 * pairs["1w"] * (p ** 4 - p ** 6))


def vsamp_variance(b_all: np.ndarray, q: np.ndarray | None = None) -> float:
    """Exact variance of one VSamp draw b_v / (4 q(v)), q uniform if None (Lemma 4 setting).

    Var = sum_v b_v^2 / (16 q(v)) - B^2 with B = sum_v b_v / 4."""
    b = np.asarray(b_all, dtype=np.float64)
    n = b.size
    if q is None:
        q = np.full(n, 1.0 / n)
    B = b.sum() / 4.0
    return float(np.sum(b * b / (16.0 * q)) - B * B)


def wedges(u, v, nU, nV):
    """Every wedge of the graph, by enumeration (tiny graphs): a list of
    (centre population index, endpoint, endpoint, beta) with the endpoints an
    unordered pair of distinct neighbours of the centre and beta = the number
    of butterflies that contain the wedge (common neighbours of the endpoints
    other than the centre)."""
    u = np.asarray(u, np.int64)
    v = np.asarray(v, np.int64)
    nb = [[set() for _ in range(nU)], [set() for _ in range(nV)]]
    for a, x in zip(u.tolist(), v.tolist()):
        nb[0][a].add(x)
        nb[1][x].add(a)
    out = []
    for s, n in ((0, nU), (1, nV)):
        for c in range(n):
            for p, q in itertools.combinations(sorted(nb[s][c]), 2):
                common = nb[1 - s][p] & nb[1 - s][q]
                out.append((c if s == 0 else nU + c, p, q, len(common) - 1))
    return out


def esamp_term_variance(be: np.ndarray, dA: np.ndarray, dX: np.ndarray, reps: int) -> float:
    """Exact variance of one ESamp term (Algorithm 5): with exact counts
    (reps = 0) the term is b_e m / 4 for a uniform edge e; with Algorithm 7
    repeated reps times it is (m / 4) d_a d_x h / reps, h ~ Binomial(reps,
    b_e / (d_a d_x)) given e, which adds E_e[(m/4)^2 (b_e d_a d_x - b_e^2) / reps]
    (Lemma on Algorithm 7: Var = b_e d_a d_x - b_e^2 for one repetition)."""
    b = np.asarray(be, np.float64)
    m = b.size
    B = b.sum() / 4.0
    var = (m / 16.0) * np.sum(b * b) - B * B
    if reps:
        dd = np.asarray(dA, np.float64) * np.asarray(dX, np.float64)
        var += (m / 16.0) * np.sum(b * dd - b * b) / reps
    return float(var)


def mixture_q(weights: np.ndarray) -> np.ndarray:
    """q(i) = 1/(2n) + w_i / (2 W): the half-uniform mixture of the weighted VSamp draw."""
    w = np.asarray(weights, dtype=np.float64)
    n = w.size
    return 0.5 / n + 0.5 * w / w.sum()
