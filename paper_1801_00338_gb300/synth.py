"""Seeded synthetic bipartite graphs (input generation only).

This module produces the edge lists that both the CUDA path and the CPU
oracle consume.  It holds none of the butterfly-counting arithmetic: it only
draws vertex pairs.  The paper evaluates on KONECT affiliation networks
(Section 2, "Networks and Experimental Setup", Table 1); those are not
available, so the generators below stand in for them with the same shapes:
uniform bipartite graphs and Chung-Lu power-law bipartite graphs with
distinct edges, plus batches of uneven small graphs.

Randomness is counter based: the k-th output (k >= 1) of a SplitMix64
sequence seeded with s is mix64(s + k * 0x9E3779B97F4A7C15), as defined by
Steele, Lea and Flood, "Fast splittable pseudorandom number generators"
(OOPSLA 2014).  Every draw is therefore a pure function of (seed, index) and
the same graph comes out on any machine.

Edges are returned in draw order (not sorted) as two uint32 arrays (u, v) with
u in [0, nU) on the left side L = U and v in [0, nV) on the right side R = V.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def mix64(z: np.ndarray) -> np.ndarray:
    """SplitMix64 output function (Stafford's variant 13 finaliser)."""
    z = np.asarray(z, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Outputs start+1 .. start+count of the SplitMix64 sequence seeded by seed."""
    k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        return mix64(np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GAMMA)


def substream_seed(seed: int, stream: int) -> int:
    """Seed of an independent sub-stream: output number stream+1 of seed's sequence."""
    return int(splitmix64(seed, stream, 1)[0])


def uniform01(seed: int, start: int, count: int) -> np.ndarray:
    """Doubles in [0, 1) from the top 53 bits of each SplitMix64 output."""
    return (splitmix64(seed, start, count) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)


# ----------------------------------------------------------------------------
# degree weights
# ----------------------------------------------------------------------------

def _capped_pareto_mean(xmin: float, alpha: float, cap: float) -> float:
    """E[min(X, cap)] for X ~ Pareto(xmin, alpha), i.e. xmin + int_xmin^cap (xmin/x)^alpha dx."""
    if xmin >= cap:
        return cap
    if abs(alpha - 1.0) < 1e-12:
        return xmin + xmin * math.log(cap / xmin)
    return xmin + xmin ** alpha * (cap ** (1.0 - alpha) - xmin ** (1.0 - alpha)) / (1.0 - alpha)


def pareto_weights(n: int, gamma: float, mean: float, cap: float, seed: int) -> np.ndarray:
    """Expected degrees with density P(d) ~ d^-gamma (Pareto shape gamma-1), capped.

    xmin is solved by bisection so that the capped mean equals `mean`; this
    also covers gamma <= 2, where the uncapped mean does not exist.
    """
    alpha = gamma - 1.0
    if alpha <= 0:
        raise ValueError("gamma must exceed 1")
    lo, hi = 1e-9, float(mean)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if _capped_pareto_mean(mid, alpha, cap) < mean:
            lo = mid
        else:
            hi = mid
    xmin = 0.5 * (lo + hi)
    u = uniform01(seed, 0, n)
    w = xmin * np.power(1.0 - u, -1.0 / alpha)
    return np.minimum(w, cap)


# ----------------------------------------------------------------------------
# edge draws
# ----------------------------------------------------------------------------

def _draw_distinct(m: int, nU: int, nV: int, draw_pairs, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """Draw pairs in rounds until m distinct ones exist; keep the first m distinct in draw order."""
    import torch  # multi-threaded CPU sort; integer keys only, so the result is deterministic
    if m > nU * nV:
        raise ValueError("more edges requested than vertex pairs")
    keys = torch.empty(0, dtype=torch.int64)
    rnd = 0
    have = 0
    while have < m:
        batch = int((m - have) * 1.15) + 1024
        a, x = draw_pairs(substream_seed(seed, 2 * rnd), substream_seed(seed, 2 * rnd + 1), batch)
        new = torch.from_numpy(a.astype(np.int64) * nV + x.astype(np.int64))
        keys = torch.cat([keys, new])
        srt, order = torch.sort(keys, stable=True)
        first = torch.ones_like(srt, dtype=torch.bool)
        first[1:] = srt[1:] != srt[:-1]
        first_idx = order[first]
        have = int(first_idx.numel())
        rnd += 1
        if rnd > 400:
            raise RuntimeError("edge generator did not reach m distinct edges")
    first_idx, _ = torch.sort(first_idx)
    sel = keys[first_idx[:m]].numpy()
    u = (sel // nV).astype(np.uint32)
    v = (sel % nV).astype(np.uint32)
    return u, v


def _pick(bits: np.ndarray, n: int) -> np.ndarray:
    """Uniform index in [0, n) from the high 32 bits (multiply-high, Lemire 2019)."""
    return (((bits >> np.uint64(32)) * np.uint64(n)) >> np.uint64(32)).astype(np.int64)


def uniform_bipartite(nU: int, nV: int, m: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """m distinct edges drawn uniformly from U x V (duplicates rejected)."""
    def draw(s1, s2, cnt):
        return _pick(splitmix64(s1, 0, cnt), nU), _pick(splitmix64(s2, 0, cnt), nV)
    return _draw_distinct(m, nU, nV, draw, seed)


def chung_lu_bipartite(nU: int, nV: int, m: int, gamma_u: float, gamma_v: float,
                       seed: int, cap: float = 2.0e5) -> tuple[np.ndarray, np.ndarray]:
    """Chung-Lu bipartite graph: endpoints drawn proportionally to Pareto weights.

    Each side's expected degrees follow a capped Pareto law with density
    exponent gamma and mean m/|side|.  Pairs (a, x) are drawn with probability
    proportional to w_a * w_x and duplicates are rejected until exactly m
    distinct edges exist.
    """
    wU = pareto_weights(nU, gamma_u, m / nU, min(cap, nV), substream_seed(seed, 1001))
    wV = pareto_weights(nV, gamma_v, m / nV, min(cap, nU), substream_seed(seed, 1002))
    cU = np.cumsum(wU)
    cV = np.cumsum(wV)
    import torch
    tU = torch.from_numpy(cU)
    tV = torch.from_numpy(cV)

    def draw(s1, s2, cnt):
        import torch
        a = torch.searchsorted(tU, torch.from_numpy(uniform01(s1, 0, cnt) * cU[-1]), right=True).numpy()
        x = torch.searchsorted(tV, torch.from_numpy(uniform01(s2, 0, cnt) * cV[-1]), right=True).numpy()
        return np.minimum(a, nU - 1), np.minimum(x, nV - 1)
    return _draw_distinct(m, nU, nV, draw, substream_seed(seed, 1003))


def complete_bipartite(a: int, b: int) -> tuple[np.ndarray, np.ndarray]:
    """K_{a,b}: every pair of U = [0, a) and V = [0, b)."""
    u = np.repeat(np.arange(a, dtype=np.uint32), b)
    v = np.tile(np.arange(b, dtype=np.uint32), a)
    return u, v


@dataclass
class Graph:
    """An edge list with its side sizes."""
    u: np.ndarray
    v: np.ndarray
    nU: int
    nV: int

    @property
    def m(self) -> int:
        return int(self.u.size)


# ----------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------

def uniform_small(seed: int = 1) -> Graph:
    """|U|=2,000, |V|=3,000, 20,000 distinct uniform edges."""
    u, v = uniform_bipartite(2000, 3000, 20000, seed)
    return Graph(u, v, 2000, 3000)


def chung_lu_1m_5m(seed: int = 2) -> Graph:
    """|U|=1M, |V|=5M, 50M distinct edges, exponents 2.1 (U) / 2.5 (V), degree cap 200k."""
    u, v = chung_lu_bipartite(1_000_000, 5_000_000, 50_000_000, 2.1, 2.5, seed)
    return Graph(u, v, 1_000_000, 5_000_000)


def chung_lu_scaled(nU: int, nV: int, m: int, gamma_u: float, gamma_v: float, seed: int,
                    cap: float = 2.0e5) -> Graph:
    u, v = chung_lu_bipartite(nU, nV, m, gamma_u, gamma_v, seed, cap)
    return Graph(u, v, nU, nV)


def uneven_batch_params(count: int, seed: int, m_lo: float = 1e3, m_hi: float = 1e6,
                        mean_degree: float = 8.0):
    """Per-graph (nU, nV, m, gamma) for a batch of uneven graphs.

    m is log-uniform in [m_lo, m_hi], |V|/|U| uniform in [0.2, 5], the
    exponent uniform in [1.9, 3.0] and |U| + |V| = 2m / mean_degree.
    """
    r = uniform01(seed, 0, 4 * count).reshape(count, 4)
    out = []
    for i in range(count):
        m = int(round(math.exp(math.log(m_lo) + r[i, 0] * (math.log(m_hi) - math.log(m_lo)))))
        ratio = 0.2 + 4.8 * r[i, 1]
        gamma = 1.9 + 1.1 * r[i, 2]
        n = max(4, int(round(2 * m / mean_degree)))
        nU = max(2, int(round(n / (1 + ratio))))
        nV = max(2, n - nU)
        while nU * nV < 2 * m:
            nU += 1
            nV += 1
        out.append((nU, nV, m, gamma))
    return out


def uneven_batch_graph(i: int, params) -> tuple[np.ndarray, np.ndarray, int, int]:
    """Graph i of a batch made by uneven_batch_params: a Chung-Lu graph with
    the same exponent on both sides, seed 100,000 + i."""
    nU, nV, m, gamma = params[i]
    u, v = chung_lu_bipartite(nU, nV, m, gamma, gamma, 100_000 + i)
    return u, v, nU, nV


def _batch_graph_job(args):
    i, params = args
    return uneven_batch_graph(i, params)


def uneven_batch(count: int, seed: int, workers: int = 0, m_lo: float = 1e3, m_hi: float = 1e6):
    """The graphs of uneven_batch_params(count, seed, m_lo, m_hi) as (u, v, nU,
    nV) tuples, made by a pool of spawned worker processes (none inherits a
    CUDA context); the graphs do not depend on the worker count."""
    import multiprocessing as mp
    import os
    params = uneven_batch_params(count, seed, m_lo, m_hi)
    jobs = [(i, params) for i in range(count)]
    workers = workers or min(16, os.cpu_count() or 1)
    if workers <= 1:
        return [_batch_graph_job(j) for j in jobs]
    with mp.get_context("spawn").Pool(workers) as pool:
        return pool.map(_batch_graph_job, jobs, chunksize=8)
