"""Autotuner of the counting path's scheduling settings (bfc.h: bfc_tuning).

The settings decide how the start vertices of Algorithm 1 are spread over the
kernels: which vertices get a warp with a shared-memory hash table and which
get a CTA with dense counter windows (the bucket thresholds), how many
top-ranked vertices go to the tensor-core hub block and at which column
density (the hash / window / MMA choice), which single-window vertices skip
the window walk, and which sweep gives the local counts.  None of them
changes a count (Lemma 1 sums over start vertices, in any grouping), only the
time.

For one graph, `autotune` times candidate settings of a workload of counting
calls by coordinate descent (one setting at a time, the others fixed, a few
timed repetitions each), checks that every candidate returns exactly the same
counts, and keeps the fastest.  The choice is cached per (GPU, graph
statistics) in a JSON file; a graph with the same statistics reuses it, and a
graph whose statistics are close (within `NEAR` in the log-space distance of
`signature`) starts from it.

The timing and counting go through the C ABI (bfc.py); `measure` may be
replaced by any function of (tuning) -> (ms, counts) for tests.
"""
from __future__ import annotations

import json
import math
import os
import statistics
from dataclasses import dataclass, field

from . import bfc

NO_HUBS = bfc.BFC_TUNE_NO_HUBS
NO_FLAT = bfc.BFC_TUNE_NO_FLAT
DEFAULT = {"warp_max_wedges": 512, "small_max_segs": 128, "hubs": 0, "tau": 0, "local_sweep": 0, "flat_max_avg": 64,
           "hl_max_light": 0}
# log-space distance under which another graph's cached choice is a starting point
NEAR = 0.25


def cache_path_default() -> str:
    p = os.environ.get("BFC_TUNE_CACHE")
    if p:
        return p
    return os.path.join(os.path.expanduser("~"), ".cache", "paper_1801_00338_gb300", "tuning.json")


def signature(stats: dict, side: int) -> dict:
    """Statistics that decide the settings: sizes, the start side's and the
    midpoint side's sum of squared degrees, and the walk's work W (Lemma 2)."""
    sq_s, sq_m = (stats["sq_u"], stats["sq_v"]) if side == 0 else (stats["sq_v"], stats["sq_u"])
    W = stats["wedges_v"] if side == 0 else stats["wedges_u"]
    return {"nU": int(stats["nU"]), "nV": int(stats["nV"]), "m": int(stats["m"]), "side": int(side),
            "sq_start": int(sq_s), "sq_mid": int(sq_m), "W": int(W)}


def _key(gpu: str, sig: dict, ops) -> str:
    return gpu + "|" + ",".join(ops) + "|" + ",".join(f"{k}={sig[k]}" for k in sorted(sig))


def distance(a: dict, b: dict) -> float:
    """Log-space distance between two signatures (inf for another start side)."""
    if a["side"] != b["side"]:
        return math.inf
    d = 0.0
    for k in ("nU", "nV", "m", "sq_start", "sq_mid", "W"):
        d = max(d, abs(math.log1p(a[k]) - math.log1p(b[k])))
    return d


def candidates(knob: str, base: dict, info: dict) -> list[int]:
    """Values tried for one setting.  info: the automatic hub count and tau of
    the graph (from bfc_exact_hub's statistics) and the start side's size."""
    if knob == "hubs":
        auto, nS = info.get("auto_hubs", 0), info.get("nS", 0)
        vals = [0, NO_HUBS]
        for f in (0.5, 2.0, 4.0):
            h = int(auto * f) // 128 * 128
            if 128 <= h <= min(bfc.BFC_HUB_MAX, nS // 128 * 128):
                vals.append(h)
        return sorted(set(vals), key=vals.index)
    if knob == "tau":
        t = info.get("auto_tau", 0)
        vals = [0] + [v for v in (t // 2, 2 * t) if v >= 2]
        return sorted(set(vals), key=vals.index)
    if knob == "small_max_segs":
        return [128, 96, 64, 32]
    if knob == "warp_max_wedges":
        return [512, 256, 128]
    if knob == "local_sweep":
        return [0, 1]
    if knob == "flat_max_avg":
        return [64, NO_FLAT, 16, 32, 128, 256]
    if knob == "hl_max_light":
        return [0, bfc.BFC_TUNE_NO_HL, 1024, 2048]
    raise ValueError(knob)


def knobs_for(ops) -> list[str]:
    """Settings that matter for a workload, the most influential first."""
    ks = []
    if "exact" in ops:
        ks += ["hubs", "tau"]
    ks += ["hl_max_light", "small_max_segs", "warp_max_wedges", "flat_max_avg"]
    if "local" in ops:
        ks += ["local_sweep"]
    return ks


@dataclass
class TuneResult:
    tuning: dict
    ms: float
    default_ms: float
    source: str                      # "cache", "search" or "search from a near graph"
    tried: list = field(default_factory=list)   # (tuning, ms) in the order timed
    counts: tuple | None = None

    def summary(self) -> dict:
        return {"tuning": self.tuning, "ms": self.ms, "default_ms": self.default_ms, "source": self.source,
                "candidates_timed": len(self.tried)}


# a candidate replaces the best setting only if it is faster by this fraction
# (timings of repeated runs vary by about a percent)
MIN_GAIN = 0.02


def coordinate_descent(measure, knobs, start: dict, info: dict, passes: int = 1, min_gain: float = MIN_GAIN):
    """Minimise measure(tuning)[0] one setting at a time, keeping a change only
    when it gains at least min_gain.  Every candidate's counts
    (measure(...)[1]) must equal the first one's; a mismatch raises, since a
    scheduling setting must never change a count."""
    best = dict(start)
    best_ms, ref_counts = measure(best)
    tried = [(dict(best), best_ms)]
    for _ in range(passes):
        improved = False
        for k in knobs:
            for val in candidates(k, best, info):
                if val == best[k]:
                    continue
                cand = dict(best)
                cand[k] = val
                ms, counts = measure(cand)
                tried.append((dict(cand), ms))
                if counts != ref_counts:
                    raise RuntimeError(f"counts differ under tuning {cand}: {counts} vs {ref_counts}")
                if ms < best_ms * (1.0 - min_gain):
                    best, best_ms, improved = cand, ms, True
        if not improved:
            break
    return best, best_ms, tried, ref_counts


def load_cache(path: str) -> dict:
    try:
        with open(path) as f:
            d = json.load(f)
        return d if isinstance(d, dict) else {}
    except (OSError, ValueError):
        return {}


def save_cache(path: str, cache: dict):
    d = os.path.dirname(path)
    if d:
        os.makedirs(d, exist_ok=True)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, path)


def lookup(cache: dict, gpu: str, sig: dict, ops):
    """(tuning, 'cache') for the same statistics; (tuning, 'near') for the
    closest graph within NEAR; (None, None) otherwise."""
    k = _key(gpu, sig, ops)
    if k in cache:
        return dict(cache[k]["tuning"]), "cache"
    best, bd = None, NEAR
    for v in cache.values():
        if v.get("gpu") != gpu or v.get("ops") != list(ops):
            continue
        d = distance(v["signature"], sig)
        if d <= bd:
            best, bd = v, d
    if best is None:
        return None, None
    return dict(best["tuning"]), "near"


def tune(measure, gpu: str, sig: dict, info: dict, ops=("exact", "local"), cache_path: str | None = None,
         use_cache: bool = True, passes: int = 1) -> TuneResult:
    """The settings for a workload `ops` on a graph with signature sig:
    the cached ones, else a coordinate-descent search (from a near graph's
    choice when there is one), stored in the cache."""
    ops = list(ops)
    path = cache_path or cache_path_default()
    cache = load_cache(path) if use_cache else {}
    hit, how = lookup(cache, gpu, sig, ops)
    if how == "cache":
        ms, counts = measure(hit)
        dms, dcounts = measure(dict(DEFAULT))
        if counts != dcounts:
            raise RuntimeError(f"counts differ under the cached tuning {hit}: {counts} vs {dcounts}")
        return TuneResult(hit, ms, dms, "cache", [(hit, ms), (dict(DEFAULT), dms)], counts)
    start = dict(DEFAULT)
    if how == "near":
        start.update(hit)
    best, best_ms, tried, counts = coordinate_descent(measure, knobs_for(ops), start, info, passes)
    default_ms = next((ms for t, ms in tried if t == DEFAULT), None)
    if default_ms is None:
        default_ms, dcounts = measure(dict(DEFAULT))
        if dcounts != counts:
            raise RuntimeError(f"counts differ under the default tuning: {dcounts} vs {counts}")
        tried.append((dict(DEFAULT), default_ms))
    if use_cache:
        cache[_key(gpu, sig, ops)] = {"gpu": gpu, "ops": ops, "signature": sig, "tuning": best, "ms": best_ms,
                                      "default_ms": default_ms}
        save_cache(path, cache)
    return TuneResult(best, best_ms, default_ms, "search" if how is None else "search from a near graph", tried,
                      counts)


# ----------------------------------------------------------------------------
# GPU measurement through the C ABI
# ----------------------------------------------------------------------------

def gpu_measure(graph: "bfc.Graph", ops=("exact", "local"), reps: int = 3, warmup: int = 1, stream=None):
    """measure(tuning) -> (median ms of the workload, counts) for a bfc.Graph.
    The workload runs the calls of `ops` back to back on one stream: "exact"
    = bfc_exact with BFC_HUB_MMA, "local" = bfc_local_counts into device
    arrays.  counts = (B of each call, and the sums of the local outputs)."""
    import torch
    s = stream or torch.cuda.current_stream()
    sp = s.cuda_stream
    L = bfc.load()
    import ctypes
    st = graph.stats
    nU, nV, m = graph.nU, graph.nV, st["m"]
    bU = torch.empty(max(nU, 1), dtype=torch.int64, device="cuda")
    bV = torch.empty(max(nV, 1), dtype=torch.int64, device="cuda")
    be = torch.empty(max(m, 1), dtype=torch.int64, device="cuda")
    Bh, side_h, B2 = ctypes.c_uint64(), ctypes.c_int(), ctypes.c_uint64()

    def run():
        out = []
        for op in ops:
            if op == "exact":
                bfc._check(L.bfc_exact(graph.h, bfc.BFC_HUB_MMA, ctypes.byref(Bh), ctypes.byref(side_h), sp),
                           "bfc_exact")
                out.append(int(Bh.value))
            elif op == "local":
                bfc._check(L.bfc_local_counts(graph.h, 0, bU.data_ptr(), bV.data_ptr(), be.data_ptr(),
                                              ctypes.byref(B2), sp), "bfc_local_counts")
                out.append(int(B2.value))
            else:
                raise ValueError(op)
        return out

    def measure(tuning: dict):
        bfc.bfc_set_tuning(graph.h, tuning)
        for _ in range(warmup):
            run()
        times = []
        for _ in range(reps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(s)
            Bs = run()
            e1.record(s)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        counts = list(Bs)
        if "local" in ops:
            counts += [int(bU[:nU].sum()), int(bV[:nV].sum()), int(be[:m].sum()),
                       int((be[:m] * torch.arange(1, m + 1, device="cuda", dtype=torch.int64)).sum())]
        return statistics.median(times), tuple(counts)

    return measure


def graph_info(graph: "bfc.Graph") -> dict:
    """The automatic hub count and tau of a graph and its start side's size."""
    B, side, hs = graph.exact_hub()
    nS = graph.nV if side else graph.nU
    return {"auto_hubs": int(hs["hubs"]), "auto_tau": int(hs["tau"]), "nS": int(nS), "side": int(side)}


def gpu_name() -> str:
    import torch
    return torch.cuda.get_device_name()


def autotune(graph: "bfc.Graph", ops=("exact", "local"), cache_path: str | None = None, use_cache: bool = True,
             reps: int = 3, passes: int = 1) -> TuneResult:
    """Tune a graph's settings for the workload `ops`, leave the chosen ones
    set on the graph and return them (see `tune`)."""
    info = graph_info(graph)
    st = dict(graph.stats)
    st.update(nU=graph.nU, nV=graph.nV)
    sig = signature(st, info["side"])
    res = tune(gpu_measure(graph, ops, reps=reps), gpu_name(), sig, info, ops, cache_path, use_cache, passes)
    bfc.bfc_set_tuning(graph.h, res.tuning)
    return res
