#!/usr/bin/env python
"""Benchmark: exact butterfly counting (B, per-vertex b_v, per-edge b_e) of the
Chung-Lu bipartite graph |U| = 1M, |V| = 5M, 50M distinct edges, exponents
2.1 (U) / 2.5 (V), on one GB300 per rank.

One step = the whole counting path on the device-resident edge list: graph
build (sort, validate, both adjacency structures), degree statistics and side
choice (Algorithm 1), rank layout and classes, ExactBFC (B, the ordered
one-sided sweep) and the ordered per-edge sweep that gives eBFC for every edge
and, through half sums of b_e over each vertex's edges, vBFC for every vertex
(bfc_local_counts).  Metric: wedges/s, where a step's wedges are
W = sum over the midpoint side of C(d, 2) (Lemma 2: the work of Algorithm 1).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl own|reference]

Under torchrun (N > 1) every rank runs the same workload on its own GPU
(replicas); value = N * W / max-over-ranks step time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "exact-count wedges/s on 1 GB300; rel. error at equal time, learned vs uniform VSamp"
WORKLOAD = "chung_lu_U1M_V5M_E50M_g2.1_2.5_seed2: ExactBFC + vBFC + eBFC"
CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


# DRAM bytes (read + write) per call of each counting-kernel set, from one ncu
# capture of the kernels' dram__bytes counters, valid only for the kernel
# source they were taken with (its SHA-256 prefix).
MEASURED_TRAFFIC = {"source_sha256": "8be147523665e5b3",
                    "bytes": {"win.edge": 17.10e9, "win.total": 5.92e9}}


def measured_traffic(tag: str):
    import hashlib
    src = os.path.join(ROOT, "paper_1801_00338_gb300", "csrc", "wedge.cu")
    with open(src, "rb") as f:
        h = hashlib.sha256(f.read()).hexdigest()[:16]
    if h != MEASURED_TRAFFIC["source_sha256"]:
        return None
    return MEASURED_TRAFFIC["bytes"].get(tag)


def max_over_ranks(x: float, dist=None) -> float:
    """The largest x over all ranks (the timing rule: the job is as slow as its
    slowest rank); x itself without a process group."""
    if dist is None:
        return x
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, units_per_rank: float, ms: float) -> float:
    """Units per second of the whole job: every rank processes units_per_rank
    (replicas, weak scaling) within the slowest rank's ms."""
    return world * units_per_rank / (ms / 1e3)


def measured_peaks(key: str = "hbm_gbs"):
    """(peak, 'measured' | 'fallback') for hbm_gbs (GB/s) or a bf16 TFLOP/s key."""
    fallback = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        if key in d:
            return float(d[key]), "measured"
    return fallback[key], "fallback"


class ClockSampler:
    """nvidia-smi samples every 200 ms during the timed region."""

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={CLOCK_FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for nm, val in zip(names, f[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def default_tuning():
    from paper_1801_00338_gb300 import autotune as AT
    return dict(AT.DEFAULT)


def workload():
    from paper_1801_00338_gb300 import synth
    return synth.chung_lu_1m_5m()


# ----------------------------------------------------------------------------
# CPU oracle timing (the baseline; never the target)
# ----------------------------------------------------------------------------

def oracle_sample(g, side: int, budget_s: float, prepared=None):
    """Time the oracle's Algorithm 1 loops over start vertices spread evenly over
    the start side until about budget_s of CPU time.  Returns (wedges/s in units
    of W, description, prepared handle)."""
    import oracle as O
    n = g.nU if side == 0 else g.nV
    P = prepared or O.Prepared(g.u, g.v, g.nU, g.nV, side)
    order = np.argsort(O_sample_keys(n)).astype(np.uint32)
    done, paths, t0 = 0, 0, time.perf_counter()
    batch = 256
    while time.perf_counter() - t0 < budget_s and done < n:
        ids = order[done:done + batch]
        _, w = P.count(ids)
        paths += w
        done += ids.size
        batch = min(batch * 2, 65536)
    dt = time.perf_counter() - t0
    # the unordered loops walk every wedge from both ends: W-units = paths / 2
    val = (paths / 2.0) / dt
    desc = (f"{done} of {n} start vertices (uniform random order, seed 7) of the same graph, "
            f"single-threaded C oracle, {paths} 2-paths in {dt:.1f} s")
    return val, desc, P


def _oracle_part(path, nU, nV, side, ids, budget_s, barrier, out):
    """One process of the all-cores oracle timing: map the edge arrays from
    the file, prepare the graph, wait for every process, then run Algorithm 1's
    loops over this process's share of the sampled start vertices for about
    budget_s seconds.  Puts (2-paths walked, vertices done, seconds)."""
    import oracle as O
    e = np.load(path, mmap_mode="r")
    P = O.Prepared(np.ascontiguousarray(e[0]), np.ascontiguousarray(e[1]), nU, nV, side)
    del e
    barrier.wait()
    done, paths, t0 = 0, 0, time.perf_counter()
    batch = 64
    while time.perf_counter() - t0 < budget_s and done < ids.size:
        part = ids[done:done + batch]
        _, w = P.count(part)
        paths += w
        done += part.size
        batch = min(batch * 2, 16384)
    out.put((paths, done, time.perf_counter() - t0))
    P.close()


def oracle_sample_all_cores(g, side: int, budget_s: float, cores: int = 0):
    """The oracle on every host core: the sampled start vertices (the same
    random order as oracle_sample) dealt round-robin to `cores` spawned
    processes, each running the single-threaded C loops on its share; the
    rate is all 2-paths over the slowest process's time.  The edge list
    reaches the processes through a temporary file.  Returns (wedges/s in
    units of W, cores, description)."""
    import multiprocessing as mp
    import shutil
    import tempfile
    # every process holds its own prepared copy of the graph (about 1.5 GB for
    # 50M edges), so at most 32 of them
    cores = cores or min(os.cpu_count() or 1, 32)
    n = g.nU if side == 0 else g.nV
    order = np.argsort(O_sample_keys(n)).astype(np.uint32)
    ctx = mp.get_context("spawn")
    tmp = tempfile.mkdtemp(prefix="bfc_oracle_")
    try:
        path = os.path.join(tmp, "edges.npy")
        np.save(path, np.stack([g.u.astype(np.uint32), g.v.astype(np.uint32)]))
        barrier, out = ctx.Barrier(cores), ctx.Queue()
        procs = [ctx.Process(target=_oracle_part, args=(path, g.nU, g.nV, side, order[i::cores].copy(), budget_s,
                                                        barrier, out))
                 for i in range(cores)]
        for pr in procs:
            pr.start()
        res = [out.get(timeout=600 + 4 * budget_s) for _ in procs]
        for pr in procs:
            pr.join()
    finally:
        shutil.rmtree(tmp, ignore_errors=True)
    paths = sum(r[0] for r in res)
    done = sum(r[1] for r in res)
    dt = max(r[2] for r in res)
    val = (paths / 2.0) / dt
    desc = (f"{done} of {n} start vertices (the same random order, dealt round-robin) on {cores} processes "
            f"of the single-threaded C oracle, {paths} 2-paths in {dt:.1f} s")
    return val, cores, desc


def O_sample_keys(n):
    from paper_1801_00338_gb300 import synth
    return synth.splitmix64(7, 0, n)


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    g = workload()
    from paper_1801_00338_gb300 import synth  # noqa: F401
    # the start side by Algorithm 1 (host arithmetic on degrees, oracle-independent of the GPU)
    dU = np.bincount(g.u, minlength=g.nU).astype(np.float64)
    dV = np.bincount(g.v, minlength=g.nV).astype(np.float64)
    side = 1 if (dU * dU).sum() < (dV * dV).sum() else 0
    mid_deg = dV if side == 0 else dU
    W = float((mid_deg * (mid_deg - 1) / 2).sum())
    P = None
    per_step = 6.0
    vals = []
    for i in range(args.warmup + args.steps):
        v, desc, P = oracle_sample(g, side, per_step, P)
        if i >= args.warmup:
            vals.append(v)
    value = statistics.median(vals)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "wedges/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": W / value * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "W": int(W)},
        "cpu_baseline": {"value": value, "unit": "wedges/s", "cores": 1, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": "wedges/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------
# the other workloads of the line (untimed by the step; each reports its own
# times, measured around whole library calls)
# ----------------------------------------------------------------------------

def extra_batch(bfc) -> dict:
    """Batched exact counting of 4,096 seeded uneven graphs (m log-uniform in
    [10^3, 10^6], side ratio in [0.2, 5], exponent in [1.9, 3.0]) in one
    bfc_exact_batch call: host edge lists in, per-graph B and side out."""
    import torch
    from paper_1801_00338_gb300 import synth
    t0 = time.perf_counter()
    graphs = synth.uneven_batch(4096, 5)
    gen_s = time.perf_counter() - t0
    edges, W = 0, 0
    for u, v, nU, nV in graphs:
        dU = np.bincount(u, minlength=nU).astype(np.float64)
        dV = np.bincount(v, minlength=nV).astype(np.float64)
        mid = dU if (dU * dU).sum() < (dV * dV).sum() else dV  # Algorithm 1: wedges centred on the other side
        W += int((mid * (mid - 1) / 2).sum())
        edges += len(u)
    bfc.bfc_exact_batch(graphs)  # warm-up
    times = []
    for _ in range(3):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        B, side = bfc.bfc_exact_batch(graphs)
        torch.cuda.synchronize()
        times.append(time.perf_counter() - t0)
    dt = float(np.median(times))
    return {"workload": "4096 uneven Chung-Lu graphs, synth.uneven_batch_params(4096, 5)", "graphs": 4096,
            "edges": edges, "W": W, "gen_s": gen_s, "s_per_call": dt, "s_all": times, "graphs_per_s": 4096 / dt,
            "edges_per_s": edges / dt, "wedges_per_s": W / dt, "B_total": int(B.astype(np.float64).sum()),
            "h2d_in_timed_call": True}


def extra_estimators(bfc) -> dict:
    """256 ESpar trials at p = 0.05 and 256 ClrSpar trials with 20 colours
    (each estimator one persistent launch) on the 20M x 40M, 300M-edge
    Chung-Lu graph (exponents 2.0 / 2.3, seed 3), against its exact count."""
    import torch
    from paper_1801_00338_gb300 import synth
    t0 = time.perf_counter()
    g = synth.chung_lu_scaled(20_000_000, 40_000_000, 300_000_000, 2.0, 2.3, 3)
    out = {"workload": "chung_lu_U20M_V40M_E300M_g2.0_2.3_seed3", "gen_s": time.perf_counter() - t0}
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        G = bfc.Graph(g.u, g.v, g.nU, g.nV, stream=stream)
    del g
    try:
        B, side = G.exact(stream=stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        B2, _ = G.exact(stream=stream)
        torch.cuda.synchronize()
        out["exact"] = {"B": int(B), "start_side": "UV"[side], "s": time.perf_counter() - t0}
        assert B2 == B
        st = G.stats
        out["exact"]["W"] = int(st["wedges_v"] if side == 0 else st["wedges_u"])
        out["exact"]["wedges_per_s"] = out["exact"]["W"] / out["exact"]["s"]
        # scheduling settings chosen by the autotuner for this graph's exact count
        from paper_1801_00338_gb300 import autotune as AT
        res = AT.autotune(G, ("exact",), use_cache=False)
        assert res.counts[0] == B
        out["tuning"] = dict(res.tuning, source="autotuner (" + res.source + ")", tuned_ms=res.ms,
                             default_ms=res.default_ms, candidates_timed=len(res.tried))
        for name, fn, arg in (("espar", G.espar, 0.05), ("clrspar", G.clrspar, 20)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            est, _ = fn(arg, 256, 2024, stream=stream)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t0
            est = np.asarray(est, np.float64)
            rel = np.abs(est - B) / B
            out[name] = {("p" if name == "espar" else "colors"): arg, "trials": 256, "launches_per_call": 1,
                         "mean": float(est.mean()), "median": float(np.median(est)),
                         "rel_err_of_mean": float(abs(est.mean() - B) / B),
                         "median_rel_err_single": float(np.median(rel)), "s_total": dt, "ms_per_trial": dt / 256 * 1e3}
    finally:
        G.close()
    return out


def extra_vsamp(bfc) -> dict:
    """The learned proposal: trained on 200 seeded Chung-Lu graphs (m
    log-uniform in [10^5, 2 x 10^7]), then uniform against learned VSamp at
    equal GPU time on the held-out 5M x 10M, 100M-edge graph."""
    import torch
    from paper_1801_00338_gb300 import learned as Ln
    from paper_1801_00338_gb300 import synth
    tr, info = Ln.train_proposal(count=200, m_lo=1e5, m_hi=2e7, steps=2000, seed=0)
    t0 = time.perf_counter()
    h = synth.chung_lu_scaled(5_000_000, 10_000_000, 100_000_000, 2.3, 2.3, 10_000)
    info["heldout_gen_s"] = time.perf_counter() - t0
    with bfc.Graph(h.u, h.v, h.nU, h.nV) as G:
        del h
        bU, bV, B = G.per_vertex()
        b = np.concatenate([bU.cpu().numpy(), bV.cpu().numpy()]).astype(np.float64)
        res = Ln.equal_time(G, b, int(B), tr.wb, trials=9, seed=7, rel=0.02)
    res["training"] = info
    res["heldout"] = {"workload": "chung_lu_U5M_V10M_E100M_g2.3_2.3_seed10000", "B": int(B)}
    return res


Z50 = 0.6744897501960817  # median of |N(0, 1)|


def _draws_for(var1: float, B: float, rel: float = 0.01) -> int:
    return max(1, int(math.ceil((Z50 / rel) ** 2 * var1 / (B * B))))


def _timed(fn):
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    out = fn()
    torch.cuda.synchronize()
    return out, time.perf_counter() - t0


def samplers_eval(g, budget_s: float = 60.0, reps: int = 1000, p_espar: float = 0.05) -> dict:
    """The sampling estimators at equal accuracy on one graph (Section 5's
    comparison): VSamp (Algorithm 4), ESamp with exact per-edge counts
    (Algorithm 5) and with Algorithm 7's estimate (1,000 repetitions), WSamp
    (Algorithm 6) and ESpar (Algorithm 8): single-draw variance (exact from the
    local counts where the lemmas give it, else empirical), draws for a 1%
    median error (normal approximation), GPU time per draw from one long call,
    and the median error of 30 trials at that draw count (capped by a time
    budget)."""
    import torch
    from paper_1801_00338_gb300 import bfc
    out = {"graph": {"nU": g.nU, "nV": g.nV, "m": g.m}}
    with bfc.Graph(g.u, g.v, g.nU, g.nV) as G:
        (B, side), t_exact = _timed(lambda: G.exact(hub_mma=True))
        (B, side), t_exact = _timed(lambda: G.exact(hub_mma=True))
        out["exact"] = {"B": int(B), "s": t_exact}
        lU, lV, le, _ = G.local_counts()
        n, m = g.nU + g.nV, g.m
        b = torch.cat([lU, lV]).to(torch.float64)
        be = le.to(torch.float64)
        # exact single-draw variances
        Bf = float(B)
        var = {"vsamp": (n / 16.0) * float((b * b).sum().item()) - Bf * Bf,
               "esamp": (m / 16.0) * float((be * be).sum().item()) - Bf * Bf}
        cu, cv = G.edges()
        dU = torch.bincount(cu.long(), minlength=g.nU).to(torch.float64)
        dV = torch.bincount(cv.long(), minlength=g.nV).to(torch.float64)
        dd = dU[cu.long()] * dV[cv.long()]
        var["esamp_fast"] = var["esamp"] + (m / 16.0) * float((be * dd - be * be).sum().item()) / reps
        del lU, lV, le, b, be, cu, cv, dd
        samplers = {
            "vsamp": lambda k, T, s: G.vsamp(k, T, s),
            "esamp": lambda k, T, s: G.esamp(k, T, s),
            "esamp_fast": lambda k, T, s: G.esamp(k, T, s, reps=reps),
            "wsamp": lambda k, T, s: G.wsamp(k, T, s),
        }
        res = {}
        for name, fn in samplers.items():
            r = {}
            # pilot: per-draw time (and the empirical variance where no exact one exists)
            k0, T0 = 4096, 64
            fn(256, 2, 1)
            est, dt = _timed(lambda: fn(k0, T0, 2))
            spd = dt / (k0 * T0)
            if name in var:
                r["var_single"] = var[name]
                r["var_kind"] = "exact"
                r["var_single_empirical"] = float(np.var(est, ddof=1) * k0)
            else:
                r["var_single"] = float(np.var(est, ddof=1) * k0)
                r["var_kind"] = "empirical (64 trials x 4096 draws)"
            kk = _draws_for(r["var_single"], B)
            r["draws_1pct"] = kk
            # the check: 30 trials at kk draws, capped by the time budget
            k_run = int(max(1, min(kk, budget_s / (30 * spd))))
            est, dt = _timed(lambda: fn(k_run, 30, 3))
            r["draws_run"] = k_run
            r["s_per_draw"] = dt / (k_run * 30)
            r["time_1pct_s"] = kk * r["s_per_draw"]
            r["median_rel_err_30"] = float(np.median(np.abs(est - B) / B))
            r["expected_median_rel_err"] = Z50 * math.sqrt(r["var_single"] / k_run) / B
            res[name] = r
        # ESpar: one trial is one "draw"
        r = {"p": p_espar}
        G.espar(p_espar, 2, 1)
        (est, beta), dt = _timed(lambda: G.espar(p_espar, 30, 4))
        est = np.asarray(est, np.float64)
        r["s_per_trial"] = dt / 30
        r["var_single"] = float(np.var(est, ddof=1))
        r["var_kind"] = "empirical (30 trials)"
        kk = _draws_for(r["var_single"], B)
        r["trials_1pct"] = kk
        r["time_1pct_s"] = kk * r["s_per_trial"]
        r["median_rel_err_single_trial"] = float(np.median(np.abs(est - B) / B))
        res["espar"] = r
        out["samplers"] = res
    return out


def run_profile_case(scale: int):
    """The benchmark's graph shrunk by `scale` (|U| = 10^6 / S, |V| = 5 x 10^6 / S,
    5 x 10^7 / S edges, the same exponents and seed): graph build,
    bfc_exact(BFC_HUB_MMA) and bfc_local_counts twice, for profilers."""
    import ctypes

    import torch

    from paper_1801_00338_gb300 import bfc, synth
    from paper_1801_00338_gb300 import build as B
    B.build()
    S = scale
    g = synth.chung_lu_scaled(1_000_000 // S, 5_000_000 // S, 50_000_000 // S, 2.1, 2.5, 2)
    du = torch.from_numpy(g.u.astype(np.int32)).cuda()
    dv = torch.from_numpy(g.v.astype(np.int32)).cuda()
    bU = torch.empty(g.nU, dtype=torch.int64, device="cuda")
    bV = torch.empty(g.nV, dtype=torch.int64, device="cuda")
    be = torch.empty(g.m, dtype=torch.int64, device="cuda")
    L = bfc.load()
    sp = torch.cuda.current_stream().cuda_stream
    Bv, B2, side = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_int()
    for _ in range(2):
        h = bfc.bfc_graph_from_edges(du, dv, g.nU, g.nV, 0, sp)
        try:
            bfc._check(L.bfc_exact(h, bfc.BFC_HUB_MMA, ctypes.byref(Bv), ctypes.byref(side), sp), "bfc_exact")
            bfc._check(L.bfc_local_counts(h, 0, bU.data_ptr(), bV.data_ptr(), be.data_ptr(), ctypes.byref(B2), sp),
                       "bfc_local_counts")
        finally:
            bfc.bfc_graph_free(h)
    torch.cuda.synchronize()
    assert Bv.value == B2.value
    print(f"profile case 1/{S}: |U|={g.nU} |V|={g.nV} m={g.m} B={Bv.value}")
    return 0


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------

def run_own(args, rank, world, local_rank):
    import torch

    from paper_1801_00338_gb300 import bfc
    from paper_1801_00338_gb300 import build as B

    B.build()
    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))

    g = workload()
    nU, nV, m = g.nU, g.nV, g.m
    du = torch.from_numpy(g.u.astype(np.int32)).cuda()
    dv = torch.from_numpy(g.v.astype(np.int32)).cuda()
    bU = torch.empty(nU, dtype=torch.int64, device="cuda")
    bV = torch.empty(nV, dtype=torch.int64, device="cuda")
    be = torch.empty(m, dtype=torch.int64, device="cuda")
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream
    L = bfc.load()
    import ctypes

    Bh = ctypes.c_uint64()
    side_h = ctypes.c_int()

    B2h = ctypes.c_uint64()

    def step():
        h = bfc.bfc_graph_from_edges(du, dv, nU, nV, 0, sptr)
        try:
            if tuning:
                bfc.bfc_set_tuning(h, tuning)
            bfc._check(L.bfc_exact(h, bfc.BFC_HUB_MMA, ctypes.byref(Bh), ctypes.byref(side_h), sptr), "bfc_exact")
            bfc._check(L.bfc_local_counts(h, 0, bU.data_ptr(), bV.data_ptr(), be.data_ptr(), ctypes.byref(B2h), sptr),
                       "bfc_local_counts")
        finally:
            bfc.bfc_graph_free(h)
        assert B2h.value == Bh.value
        return int(Bh.value), int(side_h.value)

    # statistics of the workload (not timed)
    G = bfc.Graph(du, dv, nU, nV)
    Bval, side = G.exact()
    Bhub, _, hub_stats = G.exact_hub()
    assert Bhub == Bval
    st = G.stats
    W = st["wedges_v"] if side == 0 else st["wedges_u"]
    # scheduling settings of the step's counting calls, chosen by the
    # autotuner on this graph (not timed; every candidate's counts are checked
    # equal); --no-autotune keeps the defaults
    tuning, tune_info = None, {"source": "defaults"}
    if not args.no_autotune:
        from paper_1801_00338_gb300 import autotune as AT
        res = AT.autotune(G, ("exact", "local"), use_cache=False)
        assert res.counts[0] == Bval
        tuning = res.tuning
        tune_info = {"source": "autotuner (" + res.source + ")", "tuned_ms": res.ms, "default_ms": res.default_ms,
                     "candidates_timed": len(res.tried)}
        for t, ms in res.tried:
            print(f"autotune {ms:9.3f} ms {t}", file=sys.stderr)
    if tuning and tuning["hubs"] != bfc.BFC_TUNE_NO_HUBS:
        # the hub block as the tuned step runs it (for its roofline below)
        _, _, hub_stats = G.exact_hub(hubs=min(tuning["hubs"], (nV if side else nU) // 128 * 128),
                                      tau=tuning["tau"])
    ps = G.plan_stats(side)
    G.close()

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        step()
    barrier()
    bfc.bfc_profile_reset()
    bfc.bfc_profile_enable(True)
    launches0 = bfc.bfc_launch_count()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        barrier()
    launches = bfc.bfc_launch_count() - launches0
    bfc.bfc_profile_enable(False)
    ms = e0.elapsed_time(e1) / args.steps
    prof = {t: bfc.bfc_profile_read(t) for t in bfc.PROFILE_TAGS}
    ms = max_over_ranks(ms, dist)
    value = whole_job_rate(world, W, ms)

    # ---- end to end through the C ABI with host buffers (pinned), copies timed
    hu = torch.from_numpy(g.u.astype(np.int32)).pin_memory()
    hv = torch.from_numpy(g.v.astype(np.int32)).pin_memory()
    obU = torch.empty(nU, dtype=torch.int64).pin_memory()
    obV = torch.empty(nV, dtype=torch.int64).pin_memory()
    obe = torch.empty(m, dtype=torch.int64).pin_memory()

    def e2e_step():
        hh = ctypes.c_void_p()
        bfc._check(L.bfc_graph_from_edges(hu.data_ptr(), hv.data_ptr(), m, nU, nV, 0, sptr, ctypes.byref(hh)),
                   "bfc_graph_from_edges")
        h = hh.value
        try:
            if tuning:
                bfc.bfc_set_tuning(h, tuning)
            bfc._check(L.bfc_exact(h, bfc.BFC_HUB_MMA, ctypes.byref(Bh), ctypes.byref(side_h), sptr), "bfc_exact")
            bfc._check(L.bfc_local_counts(h, 0, bU.data_ptr(), bV.data_ptr(), be.data_ptr(), ctypes.byref(B2h), sptr),
                       "bfc_local_counts")
            obU.copy_(bU, non_blocking=True)
            obV.copy_(bV, non_blocking=True)
            obe.copy_(be, non_blocking=True)
        finally:
            bfc.bfc_graph_free(h)
        torch.cuda.synchronize()

    # every end-to-end step is timed on the host (each ends with a device
    # synchronise, so its time holds its copies and its kernels); the median
    # step is reported, since host-side allocation and copy times vary
    e2e_steps = max(5, min(args.steps, 10))
    e2e_step()
    barrier()
    e2e_times = []
    for _ in range(e2e_steps):
        t0 = time.perf_counter()
        e2e_step()
        e2e_times.append((time.perf_counter() - t0) * 1e3)
    barrier()
    e2e_ms = float(np.median(e2e_times))
    e2e_ms = max_over_ranks(e2e_ms, dist)
    assert int(obU.sum()) == 2 * Bval and int(obe.sum()) == 4 * Bval

    # ---- roofline of the dominant kernel
    peak, peak_kind = measured_peaks()
    dom = max((t for t in prof if t.split(".")[0] in bfc.TAG_CLASSES), key=lambda t: prof[t][1])
    n_launch, tot_ms = prof[dom]
    cls = dom.split(".")[0]
    mode = dom.split(".")[1]
    wedges = sum(ps["work"][c] for c in bfc.TAG_CLASSES[cls])
    rows = sum(ps["rows"][c] for c in bfc.TAG_CLASSES[cls])
    if mode in ("local", "single"):
        # whole rows: every wedge is walked from both ends
        wedges = 2 * wedges
    per_wedge = 8 if mode in ("edge", "local") else 4
    alg_bytes = per_wedge * wedges + 16 * rows
    avg_ms = tot_ms / max(n_launch, 1)
    achieved = alg_bytes / (avg_ms / 1e3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": measured_traffic(dom), "kernel": {"warp": "k_warp_class", "win": "k_cta_win", "big": "k_cta_big"}[cls] + f"<{mode}>", "peak_kind": peak_kind,
                "alg_bytes_per_launch": alg_bytes, "avg_launch_ms": avg_ms}

    # the hub block's tile kernel: upper-triangle 128 x 128 tiles over K padded to 64
    nt = hub_stats["hubs"] // 128
    Kp = max(64, -(-hub_stats["K"] // 64) * 64)
    hub_flops = nt * (nt + 1) // 2 * 128 * 128 * Kp * 2
    hn, hms = prof.get("hub.total", (0, 0.0))
    hub_roof = None
    if hn and hms > 0:
        tpk, tkind = measured_peaks("bf16_tflops_sustained")  # timed inside the long step
        ach = hub_flops / (hms / hn / 1e3) / 1e12
        hub_roof = {"bound": "tensor", "kernel": "k_hub_mma", "achieved": ach, "peak": tpk, "unit": "TFLOP/s",
                    "frac": ach / tpk, "peak_kind": tkind, "flops_per_launch": hub_flops, "avg_launch_ms": hms / hn,
                    "hubs": hub_stats["hubs"], "K": hub_stats["K"], "tau": hub_stats["tau"],
                    "light_pairs": hub_stats["light_pairs"]}

    line = {
        "metric": METRIC, "value": value, "unit": "wedges/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "nU": nU, "nV": nV, "m": m, "W": W, "B": Bval, "start_side": "UV"[side],
                   "parallelism": f"replicas{world}", "l2": "inputs larger than L2 (edge list 400 MB)",
                   "classes": ps["count"], "class_wedges": ps["work"],
                   "tuning": dict(tuning or default_tuning(), **tune_info)},
        "e2e": {"value": whole_job_rate(world, W, e2e_ms), "unit": "wedges/s", "ms_per_step": e2e_ms,
                "ms_per_step_min_max": [min(e2e_times), max(e2e_times)], "steps_timed": e2e_steps,
                "h2d_bytes_per_step": 8 * m, "d2h_bytes_per_step": 8 * (nU + nV + m) + 16},
        "gpu_launches": launches,
        "clocks": clk.summary(),
        "roofline": roofline,
        "roofline_hub_block": hub_roof,
        "kernels_ms_per_step": {t: prof[t][1] / args.steps for t in prof if prof[t][0]},
    }
    if rank == 0 and not args.no_cpu_baseline:
        v, desc, P = oracle_sample(g, side, args.cpu_budget)
        P.close()
        line["cpu_baseline"] = {"value": v, "unit": "wedges/s", "cores": 1, "kind": "oracle", "sample": desc}
        if args.cpu_all_cores:
            # a second, all-cores figure; the bench line stands without it
            try:
                va, cores, desca = oracle_sample_all_cores(g, side, args.cpu_budget)
                line["cpu_baseline"]["all_cores"] = {"value": va, "unit": "wedges/s", "cores": cores,
                                                     "kind": "oracle", "sample": desca}
            except Exception as e:  # noqa: BLE001
                line["cpu_baseline"]["all_cores"] = {"unavailable": f"{type(e).__name__}: {e}"[:200]}
    if rank == 0 and args.extras:
        # the other workloads (each failure is reported in its key, the line stands)
        del du, dv, bU, bV, be, hu, hv, obU, obV, obe
        torch.cuda.empty_cache()
        for key, fn in (("batch", extra_batch), ("estimators", extra_estimators), ("vsamp_equal_time", extra_vsamp)):
            t0 = time.perf_counter()
            try:
                line[key] = fn(bfc)
            except Exception as e:  # noqa: BLE001
                line[key] = {"unavailable": f"{type(e).__name__}: {e}"[:300]}
            line[key]["wall_s"] = time.perf_counter() - t0
            print(f"{key}: {time.perf_counter() - t0:.0f} s", file=sys.stderr, flush=True)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("own", "reference"), default="own")
    ap.add_argument("--cpu-budget", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-all-cores", action=argparse.BooleanOptionalAction, default=True,
                    help="also time the oracle on every host core (spawned processes)")
    ap.add_argument("--no-autotune", action="store_true", help="count with the default scheduling settings")
    ap.add_argument("--extras", action=argparse.BooleanOptionalAction, default=True,
                    help="also run the batched-graph, sparsification-estimator and learned-VSamp workloads")
    ap.add_argument("--samplers-eval", action="store_true",
                    help="only compare the sampling estimators at equal accuracy on the benchmark graph and exit")
    ap.add_argument("--profile-case", type=int, default=0, metavar="S",
                    help="only run the benchmark graph shrunk by S twice (for profilers) and exit")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus if args.gpus == 1 else 1)))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.profile_case:
        return run_profile_case(args.profile_case)
    if args.samplers_eval:
        from paper_1801_00338_gb300 import build as B
        from paper_1801_00338_gb300 import synth
        B.build()
        print(json.dumps(samplers_eval(synth.chung_lu_1m_5m(), budget_s=60.0)), flush=True)
        return 0
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_own(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
