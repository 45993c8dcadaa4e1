"""Thin ctypes binding of libbfc.so (include/bfc.h).

Argument marshalling only: every step of the counting path runs in the CUDA
library.  The functions keep the C names (bfc_graph_from_edges, bfc_exact,
...); :class:`Graph` wraps a handle for convenience.  There is no fallback: if
the library is missing or fails to load, every call raises.

Device arrays are torch CUDA tensors (torch is used for device memory and
streams only).  uint64 counts are returned in int64 tensors holding the same
bits (every count here is below 2^63).
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbfc.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "bfc.h")

BFC_OK = 0
BFC_INPUT_DEVICE = 0x1
BFC_DEDUP = 0x2
BFC_SIDE_AUTO = 0x0
BFC_SIDE_U = 0x10
BFC_SIDE_V = 0x20
BFC_WHOLE_ROWS = 0x100
BFC_HUB_MMA = 0x200
BFC_HUB_MAX = 16384
BFC_TUNE_NO_HUBS = 0xFFFFFFFF
BFC_TUNE_NO_FLAT = 0xFFFFFFFF
BFC_TUNE_NO_HL = 0xFFFFFFFF
TUNING_FIELDS = ("warp_max_wedges", "small_max_segs", "hubs", "tau", "local_sweep", "flat_max_avg", "hl_max_light")


class bfc_tuning(ctypes.Structure):
    _fields_ = [(f, ctypes.c_uint32) for f in TUNING_FIELDS]

_lib = None


class BfcError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {strerror(code)} ({code})")


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libbfc.so; raise if it is not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it first (python -m paper_1801_00338_gb300.build)")
    L = ctypes.CDLL(path)
    P, u32, u64, i32, dbl = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int, ctypes.c_double
    sig = {
        "bfc_graph_from_edges": [P, P, u64, u32, u32, u32, P, P],
        "bfc_graph_free": [P],
        "bfc_graph_from_csr": [P, P, u32, P, P, P, u32, P, P],
        "bfc_trim_memory": [],
        "bfc_graph_stats": [P, P, P, P, P, P],
        "bfc_graph_edges": [P, P, P, P],
        "bfc_exact": [P, u32, P, P, P],
        "bfc_exact_hub": [P, u32, u32, u32, P, P, P, P],
        "bfc_per_vertex": [P, u32, P, P, P, P],
        "bfc_per_edge": [P, u32, P, P, P],
        "bfc_local_counts": [P, u32, P, P, P, P, P],
        "bfc_espar": [P, dbl, u32, u64, P, P, P],
        "bfc_clrspar": [P, u32, u32, u64, P, P, P],
        "bfc_vsamp": [P, u64, P, u32, u64, P, P, P, P],
        "bfc_esamp": [P, u64, u32, u32, u64, P, P, P, P],
        "bfc_wsamp": [P, u64, u32, u64, P, P, P, P],
        "bfc_median_of_means": [P, u64, u32, P],
        "bfc_mom_sizes": [dbl, dbl, dbl, dbl, P, P],
        "bfc_proposal_from_weights": [P, P, u32, P, P],
        "bfc_proposal_free": [P],
        "bfc_proposal_weights": [P, P, u64, P],
        "bfc_exact_csr_noalloc": [P, P, u32, P, P, u32, u32, P, P],
        "bfc_exact_batch": [P, P, P, P, P, u32, u32, P, P, P],
        "bfc_features": [P, P, P],
        "bfc_mlp_targets": [P, u64, P, P],
        "bfc_mlp_forward": [P, P, u64, P, P],
        "bfc_mlp_grad": [P, P, P, P, u64, P, P, P],
        "bfc_mlp_adam": [P, P, P, P, P, u32, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, u32, P],
        "bfc_mlp_to_bf16": [P, P, u32, P],
        "bfc_proposal_from_scores": [P, P, P, P],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = i32
    for name in ("bfc_set_tuning", "bfc_get_tuning"):
        f = getattr(L, name)
        f.argtypes = [P, ctypes.POINTER(bfc_tuning)]
        f.restype = i32
    L.bfc_fail_alloc_after.argtypes = [ctypes.c_int64]
    L.bfc_fail_alloc_after.restype = i32
    L.bfc_set_wait_limit.argtypes = [ctypes.c_uint64]
    L.bfc_set_wait_limit.restype = i32
    L.bfc_plan_stats.argtypes = [P, i32, P, P]
    L.bfc_plan_stats.restype = i32
    L.bfc_profile_enable.argtypes = [i32]
    L.bfc_profile_enable.restype = i32
    L.bfc_profile_reset.argtypes = []
    L.bfc_profile_reset.restype = i32
    L.bfc_profile_read.argtypes = [ctypes.c_char_p, P, P]
    L.bfc_profile_read.restype = i32
    L.bfc_strerror.argtypes = [i32]
    L.bfc_strerror.restype = ctypes.c_char_p
    L.bfc_launch_count.argtypes = []
    L.bfc_launch_count.restype = u64
    _lib = L
    return L


def header_symbols(path: str = HEADER) -> list[str]:
    """Every function the public header declares."""
    txt = open(path).read()
    return sorted(set(re.findall(r"^\s*(?:int|const char \*|uint64_t)\s*(bfc_\w+)\s*\(", txt, re.M)))


def strerror(code: int) -> str:
    return load().bfc_strerror(code).decode()


def _check(rc: int, what: str):
    if rc != BFC_OK:
        raise BfcError(rc, what)


def _stream_ptr(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream or None
    if isinstance(stream, int):
        return stream or None
    return stream.cuda_stream or None


def _dptr(t) -> int:
    return t.data_ptr()


def bfc_fail_alloc_after(n: int):
    """Make the library's (n+1)-th next device allocation fail (n < 0: none)."""
    _check(load().bfc_fail_alloc_after(int(n)), "bfc_fail_alloc_after")


def bfc_set_wait_limit(ns: int):
    """Give-up limit (ns of GPU time) of the hub kernel's device waits; 0 = built-in."""
    _check(load().bfc_set_wait_limit(int(ns)), "bfc_set_wait_limit")


def bfc_trim_memory():
    _check(load().bfc_trim_memory(), "bfc_trim_memory")


def bfc_launch_count() -> int:
    return int(load().bfc_launch_count())


CLASSES = ("skip", "warp", "s2", "s4", "s8", "s6", "s5", "l2", "l4", "l8", "l16", "l10", "big")


def bfc_plan_stats(h: int, side: int, stream=None) -> dict:
    """Per-class vertex counts, wedges and start-row entries of a start side's layout."""
    out = np.zeros(41, np.uint64)
    _check(load().bfc_plan_stats(h, side, out.ctypes.data, _stream_ptr(stream)), "bfc_plan_stats")
    o = [int(x) for x in out]
    n = len(CLASSES)
    return {"nS": o[0], "count": dict(zip(CLASSES, o[1:1 + n])), "work": dict(zip(CLASSES, o[1 + n:1 + 2 * n])),
            "rows": dict(zip(CLASSES, o[1 + 2 * n:1 + 3 * n])), "W": o[1 + 3 * n]}


def bfc_profile_enable(on: bool = True):
    _check(load().bfc_profile_enable(1 if on else 0), "bfc_profile_enable")


def bfc_profile_reset():
    _check(load().bfc_profile_reset(), "bfc_profile_reset")


def bfc_profile_read(tag: str) -> tuple[int, float]:
    n = ctypes.c_uint64()
    ms = ctypes.c_double()
    _check(load().bfc_profile_read(tag.encode(), ctypes.byref(n), ctypes.byref(ms)), "bfc_profile_read")
    return int(n.value), float(ms.value)


PROFILE_TAGS = [f"{c}.{m}" for c in ("warp", "win", "big") for m in ("total", "edge", "single", "local")]
PROFILE_TAGS += ["hub.total", "hub.degree", "hub.light", "esamp.exact", "esamp.fast", "wsamp"]
# the window kernels also per class: "win.edge.s8" (8-bit counters, the 128-thread CTAs)
WIN_CLASS_TAGS = [f"win.{m}.{c}" for m in ("total", "edge", "single", "local")
                  for c in ("s2", "s4", "s8", "s6", "s5", "l2", "l4", "l8", "l16", "l10")]
# kernel tag -> the classes it runs
TAG_CLASSES = {"warp": ("warp",), "win": ("s2", "s4", "s8", "s6", "s5", "l2", "l4", "l8", "l16", "l10"),
               "big": ("big",)}


# ----------------------------------------------------------------------------
# C-named entry points
# ----------------------------------------------------------------------------

def bfc_graph_from_edges(u, v, nU: int, nV: int, flags: int = 0, stream=None) -> int:
    """Build a graph; u, v are host numpy uint32 arrays or CUDA uint32/int32 tensors."""
    L = load()
    h = ctypes.c_void_p()
    if hasattr(u, "is_cuda") and u.is_cuda:
        import torch
        if u.dtype not in (torch.int32, torch.uint32) or v.dtype != u.dtype:
            raise TypeError("device edge arrays must be int32/uint32 tensors")
        u = u.contiguous()
        v = v.contiguous()
        m = u.numel()
        rc = L.bfc_graph_from_edges(_dptr(u), _dptr(v), m, nU, nV, flags | BFC_INPUT_DEVICE, _stream_ptr(stream),
                                    ctypes.byref(h))
    else:
        u = np.ascontiguousarray(u, dtype=np.uint32)
        v = np.ascontiguousarray(v, dtype=np.uint32)
        if u.size != v.size:
            raise ValueError("u and v differ in length")
        rc = L.bfc_graph_from_edges(u.ctypes.data, v.ctypes.data, u.size, nU, nV, flags & ~BFC_INPUT_DEVICE,
                                    _stream_ptr(stream), ctypes.byref(h))
    _check(rc, "bfc_graph_from_edges")
    return h.value


def bfc_graph_from_csr(offU, nbrU, nU: int, offV, nbrV, nV: int, eidV=None, stream=None) -> int:
    """Build a graph from device rows (int64 offsets, int32 ids as CUDA tensors)."""
    h = ctypes.c_void_p()
    _check(load().bfc_graph_from_csr(_dptr(offU), _dptr(nbrU), nU, _dptr(offV), _dptr(nbrV),
                                     _dptr(eidV) if eidV is not None else None, nV, _stream_ptr(stream),
                                     ctypes.byref(h)), "bfc_graph_from_csr")
    return h.value


def bfc_set_tuning(h: int, tuning: dict | None):
    """Scheduling settings of a graph (bfc.h: bfc_tuning); None restores the
    defaults, a missing key means 0 (the default)."""
    if tuning is None:
        _check(load().bfc_set_tuning(h, None), "bfc_set_tuning")
        return
    unknown = set(tuning) - set(TUNING_FIELDS)
    if unknown:
        raise ValueError(f"unknown tuning fields {sorted(unknown)}")
    t = bfc_tuning(*[int(tuning.get(f, 0)) for f in TUNING_FIELDS])
    _check(load().bfc_set_tuning(h, ctypes.byref(t)), "bfc_set_tuning")


def bfc_get_tuning(h: int) -> dict:
    t = bfc_tuning()
    _check(load().bfc_get_tuning(h, ctypes.byref(t)), "bfc_get_tuning")
    return {f: int(getattr(t, f)) for f in TUNING_FIELDS}


def bfc_graph_free(h: int):
    _check(load().bfc_graph_free(h), "bfc_graph_free")


def bfc_graph_stats(h: int) -> dict:
    vals = [ctypes.c_uint64() for _ in range(5)]
    _check(load().bfc_graph_stats(h, *[ctypes.byref(x) for x in vals]), "bfc_graph_stats")
    keys = ("m", "sq_u", "sq_v", "wedges_u", "wedges_v")
    return {k: int(x.value) for k, x in zip(keys, vals)}


def bfc_graph_edges(h: int, m: int, stream=None):
    import torch
    u = torch.empty(m, dtype=torch.int32, device="cuda")
    v = torch.empty(m, dtype=torch.int32, device="cuda")
    _check(load().bfc_graph_edges(h, _dptr(u), _dptr(v), _stream_ptr(stream)), "bfc_graph_edges")
    return u, v


def bfc_exact(h: int, flags: int = 0, stream=None) -> tuple[int, int]:
    B = ctypes.c_uint64()
    side = ctypes.c_int()
    _check(load().bfc_exact(h, flags, ctypes.byref(B), ctypes.byref(side), _stream_ptr(stream)), "bfc_exact")
    return int(B.value), int(side.value)


def bfc_exact_hub(h: int, flags: int = 0, hubs: int = 0, tau: int = 0, stream=None) -> tuple[int, int, dict]:
    """ExactBFC with the tensor-core hub block; returns (B, start side, stats)."""
    B = ctypes.c_uint64()
    side = ctypes.c_int()
    st = (ctypes.c_uint64 * 4)()
    _check(load().bfc_exact_hub(h, flags, hubs, tau, ctypes.byref(B), ctypes.byref(side), st, _stream_ptr(stream)),
           "bfc_exact_hub")
    return int(B.value), int(side.value), dict(zip(("hubs", "K", "tau", "light_pairs"), (int(x) for x in st)))


def bfc_per_vertex(h: int, nU: int, nV: int, flags: int = 0, stream=None):
    import torch
    bU = torch.empty(nU, dtype=torch.int64, device="cuda")
    bV = torch.empty(nV, dtype=torch.int64, device="cuda")
    B = ctypes.c_uint64()
    _check(load().bfc_per_vertex(h, flags, _dptr(bU), _dptr(bV), ctypes.byref(B), _stream_ptr(stream)),
           "bfc_per_vertex")
    return bU, bV, int(B.value)


def bfc_per_edge(h: int, m: int, flags: int = 0, stream=None):
    import torch
    be = torch.empty(max(m, 1), dtype=torch.int64, device="cuda")
    B = ctypes.c_uint64()
    _check(load().bfc_per_edge(h, flags, _dptr(be), ctypes.byref(B), _stream_ptr(stream)), "bfc_per_edge")
    return be[:m], int(B.value)


def bfc_local_counts(h: int, nU: int, nV: int, m: int, flags: int = 0, stream=None):
    import torch
    bU = torch.empty(nU, dtype=torch.int64, device="cuda")
    bV = torch.empty(nV, dtype=torch.int64, device="cuda")
    be = torch.empty(max(m, 1), dtype=torch.int64, device="cuda")
    B = ctypes.c_uint64()
    _check(load().bfc_local_counts(h, flags, _dptr(bU), _dptr(bV), _dptr(be), ctypes.byref(B), _stream_ptr(stream)),
           "bfc_local_counts")
    return bU, bV, be[:m], int(B.value)


def bfc_espar(h: int, p: float, trials: int, seed: int, stream=None):
    est = np.zeros(trials, np.float64)
    beta = np.zeros(trials, np.uint64)
    _check(load().bfc_espar(h, p, trials, seed & 0xFFFFFFFFFFFFFFFF, est.ctypes.data, beta.ctypes.data,
                            _stream_ptr(stream)), "bfc_espar")
    return est, beta


def bfc_clrspar(h: int, colors: int, trials: int, seed: int, stream=None):
    est = np.zeros(trials, np.float64)
    beta = np.zeros(trials, np.uint64)
    _check(load().bfc_clrspar(h, colors, trials, seed & 0xFFFFFFFFFFFFFFFF, est.ctypes.data, beta.ctypes.data,
                              _stream_ptr(stream)), "bfc_clrspar")
    return est, beta


def bfc_proposal_from_weights(h: int, weights, stream=None) -> int:
    L = load()
    p = ctypes.c_void_p()
    if hasattr(weights, "is_cuda") and weights.is_cuda:
        rc = L.bfc_proposal_from_weights(h, _dptr(weights.contiguous()), BFC_INPUT_DEVICE, _stream_ptr(stream),
                                         ctypes.byref(p))
    else:
        w = np.ascontiguousarray(weights, dtype=np.uint32)
        rc = L.bfc_proposal_from_weights(h, w.ctypes.data, 0, _stream_ptr(stream), ctypes.byref(p))
    _check(rc, "bfc_proposal_from_weights")
    return p.value


def bfc_proposal_weights(p: int, n: int):
    """(weights as a uint32 numpy array of n entries, their sum W)."""
    w = np.zeros(n, np.uint32)
    W = ctypes.c_uint64()
    _check(load().bfc_proposal_weights(p, w.ctypes.data, n, ctypes.byref(W)), "bfc_proposal_weights")
    return w, W.value


def bfc_proposal_free(p: int):
    _check(load().bfc_proposal_free(p), "bfc_proposal_free")


def bfc_vsamp(h: int, k: int, trials: int, seed: int, proposal: int | None = None, want_draws: bool = False,
              stream=None):
    import torch
    est = np.zeros(trials, np.float64)
    drawn = bd = None
    pd = pb = None
    if want_draws:
        drawn = torch.empty(max(trials * k, 1), dtype=torch.int64, device="cuda")
        bd = torch.empty(max(trials * k, 1), dtype=torch.int64, device="cuda")
        pd, pb = _dptr(drawn), _dptr(bd)
    _check(load().bfc_vsamp(h, k, proposal, trials, seed & 0xFFFFFFFFFFFFFFFF, est.ctypes.data, pd, pb,
                            _stream_ptr(stream)), "bfc_vsamp")
    if want_draws:
        return est, drawn[: trials * k], bd[: trials * k]
    return est


def bfc_esamp(h: int, k: int, reps: int, trials: int, seed: int, want_draws: bool = False, stream=None):
    """ESamp (Algorithm 5): per-trial estimates; with want_draws also the
    device arrays of drawn canonical edges and of the draws' values (b_e, or
    Algorithm 7's hit counts when reps > 0)."""
    import torch
    est = np.zeros(trials, np.float64)
    ed = vd = None
    pe = pv = None
    if want_draws:
        ed = torch.empty(max(trials * k, 1), dtype=torch.int64, device="cuda")
        vd = torch.empty(max(trials * k, 1), dtype=torch.int64, device="cuda")
        pe, pv = _dptr(ed), _dptr(vd)
    _check(load().bfc_esamp(h, k, reps, trials, seed & 0xFFFFFFFFFFFFFFFF, est.ctypes.data, pe, pv,
                            _stream_ptr(stream)), "bfc_esamp")
    if want_draws:
        return est, ed[: trials * k], vd[: trials * k]
    return est


def bfc_wsamp(h: int, k: int, trials: int, seed: int, want_draws: bool = False, stream=None):
    """WSamp (Algorithm 6): per-trial estimates; with want_draws also the
    device arrays of centres (population index) and betas."""
    import torch
    est = np.zeros(trials, np.float64)
    cd = bd = None
    pc = pb = None
    if want_draws:
        cd = torch.empty(max(trials * k, 1), dtype=torch.int64, device="cuda")
        bd = torch.empty(max(trials * k, 1), dtype=torch.int64, device="cuda")
        pc, pb = _dptr(cd), _dptr(bd)
    _check(load().bfc_wsamp(h, k, trials, seed & 0xFFFFFFFFFFFFFFFF, est.ctypes.data, pc, pb, _stream_ptr(stream)),
           "bfc_wsamp")
    if want_draws:
        return est, cd[: trials * k], bd[: trials * k]
    return est


def bfc_median_of_means(y, groups: int) -> float:
    """Median of the means of `groups` consecutive groups of the values y."""
    y = np.ascontiguousarray(y, dtype=np.float64)
    out = ctypes.c_double()
    _check(load().bfc_median_of_means(y.ctypes.data, y.size, groups, ctypes.byref(out)), "bfc_median_of_means")
    return float(out.value)


def bfc_mom_sizes(var1: float, B: float, epsilon: float, delta: float) -> tuple[int, int]:
    """(instances per group, groups) of an (epsilon, delta) median-of-means estimate."""
    a = ctypes.c_uint64()
    g = ctypes.c_uint32()
    _check(load().bfc_mom_sizes(var1, B, epsilon, delta, ctypes.byref(a), ctypes.byref(g)), "bfc_mom_sizes")
    return int(a.value), int(g.value)


MLP_FEATURES = 6
MLP_PARAMS = 4673


def bfc_features(h: int, n: int, stream=None):
    import torch
    f = torch.empty((n, MLP_FEATURES), dtype=torch.float32, device="cuda")
    _check(load().bfc_features(h, _dptr(f), _stream_ptr(stream)), "bfc_features")
    return f


def bfc_mlp_targets(b, stream=None):
    import torch
    t = torch.empty(b.numel(), dtype=torch.float32, device="cuda")
    _check(load().bfc_mlp_targets(_dptr(b), b.numel(), _dptr(t), _stream_ptr(stream)), "bfc_mlp_targets")
    return t


def bfc_mlp_forward(w_bf16, X, stream=None):
    import torch
    y = torch.empty(X.shape[0], dtype=torch.float32, device="cuda")
    _check(load().bfc_mlp_forward(_dptr(w_bf16), _dptr(X), X.shape[0], _dptr(y), _stream_ptr(stream)),
           "bfc_mlp_forward")
    return y


def bfc_mlp_grad(w_bf16, X, T, idx=None, n=None, stream=None):
    import torch
    grad = torch.empty(MLP_PARAMS, dtype=torch.float32, device="cuda")
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    n = (idx.numel() if idx is not None else X.shape[0]) if n is None else n
    _check(load().bfc_mlp_grad(_dptr(w_bf16), _dptr(X), _dptr(T), _dptr(idx) if idx is not None else None, n,
                               _dptr(grad), _dptr(loss), _stream_ptr(stream)), "bfc_mlp_grad")
    return grad, loss


def bfc_mlp_adam(w, w_bf16, m, v, grad, lr, step, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(load().bfc_mlp_adam(_dptr(w), _dptr(w_bf16), _dptr(m), _dptr(v), _dptr(grad), MLP_PARAMS, lr, beta1, beta2,
                               eps, step, _stream_ptr(stream)), "bfc_mlp_adam")


def bfc_mlp_to_bf16(w, stream=None):
    import torch
    wb = torch.empty(MLP_PARAMS, dtype=torch.int16, device="cuda")
    _check(load().bfc_mlp_to_bf16(_dptr(w), _dptr(wb), MLP_PARAMS, _stream_ptr(stream)), "bfc_mlp_to_bf16")
    return wb


def bfc_proposal_from_scores(h: int, scores, stream=None) -> int:
    p = ctypes.c_void_p()
    _check(load().bfc_proposal_from_scores(h, _dptr(scores), _stream_ptr(stream), ctypes.byref(p)),
           "bfc_proposal_from_scores")
    return p.value


def bfc_exact_batch(graphs, stream=None):
    """B of every graph in a list of (u, v, nU, nV) host edge lists, in one pass.

    Returns (B array, start side array)."""
    G = len(graphs)
    sizes = [len(g[0]) for g in graphs]
    eoff = np.zeros(G + 1, np.uint64)
    np.cumsum(sizes, out=eoff[1:])
    u = np.ascontiguousarray(np.concatenate([np.asarray(g[0], np.uint32) for g in graphs]) if G else
                             np.zeros(0, np.uint32))
    v = np.ascontiguousarray(np.concatenate([np.asarray(g[1], np.uint32) for g in graphs]) if G else
                             np.zeros(0, np.uint32))
    nU = np.array([g[2] for g in graphs], np.uint32)
    nV = np.array([g[3] for g in graphs], np.uint32)
    B = np.zeros(G, np.uint64)
    side = np.zeros(G, np.int32)
    _check(load().bfc_exact_batch(u.ctypes.data, v.ctypes.data, eoff.ctypes.data, nU.ctypes.data, nV.ctypes.data, G,
                                  0, B.ctypes.data, side.ctypes.data, _stream_ptr(stream)), "bfc_exact_batch")
    return B, side


def bfc_exact_csr_noalloc(offU, nbrU, nU: int, offV, nbrV, nV: int, out_B, flags: int = 0, stream=None) -> int:
    """ExactBFC on device CSR tensors without allocating; out_B is a 1-element
    int64 CUDA tensor that receives B in stream order.  Returns the status code."""
    return int(load().bfc_exact_csr_noalloc(_dptr(offU), _dptr(nbrU), nU, _dptr(offV), _dptr(nbrV), nV, flags,
                                            _dptr(out_B), _stream_ptr(stream)))


# ----------------------------------------------------------------------------
# convenience wrapper
# ----------------------------------------------------------------------------

_SIDE = {None: BFC_SIDE_AUTO, "auto": BFC_SIDE_AUTO, "U": BFC_SIDE_U, "V": BFC_SIDE_V, 0: BFC_SIDE_U, 1: BFC_SIDE_V}


class Graph:
    """A bipartite graph resident on the GPU (a bfc_graph handle)."""

    def __init__(self, u, v, nU: int, nV: int, dedup: bool = False, stream=None):
        self.nU, self.nV = int(nU), int(nV)
        self.h = bfc_graph_from_edges(u, v, nU, nV, BFC_DEDUP if dedup else 0, stream)
        self.stats = bfc_graph_stats(self.h)
        self.m = self.stats["m"]

    @classmethod
    def from_csr(cls, offU, nbrU, nU: int, offV, nbrV, nV: int, eidV=None, stream=None):
        """A graph from device rows (bfc_graph_from_csr)."""
        G = cls.__new__(cls)
        G.nU, G.nV = int(nU), int(nV)
        G.h = bfc_graph_from_csr(offU, nbrU, nU, offV, nbrV, nV, eidV, stream)
        G.stats = bfc_graph_stats(G.h)
        G.m = G.stats["m"]
        return G

    def exact(self, side=None, hub_mma=False, stream=None):
        return bfc_exact(self.h, _SIDE[side] | (BFC_HUB_MMA if hub_mma else 0), stream)

    def exact_hub(self, side=None, hubs=0, tau=0, stream=None):
        return bfc_exact_hub(self.h, _SIDE[side], hubs, tau, stream)

    def per_vertex(self, side=None, whole_rows=False, stream=None):
        return bfc_per_vertex(self.h, self.nU, self.nV, _SIDE[side] | (BFC_WHOLE_ROWS if whole_rows else 0), stream)

    def per_edge(self, side=None, whole_rows=False, stream=None):
        return bfc_per_edge(self.h, self.m, _SIDE[side] | (BFC_WHOLE_ROWS if whole_rows else 0), stream)

    def local_counts(self, side=None, whole_rows=False, stream=None):
        return bfc_local_counts(self.h, self.nU, self.nV, self.m, _SIDE[side] | (BFC_WHOLE_ROWS if whole_rows else 0),
                                stream)

    def set_tuning(self, tuning: dict | None):
        bfc_set_tuning(self.h, tuning)

    def tuning(self) -> dict:
        return bfc_get_tuning(self.h)

    def plan_stats(self, side: int, stream=None):
        return bfc_plan_stats(self.h, side, stream)

    def edges(self, stream=None):
        return bfc_graph_edges(self.h, self.m, stream)

    def espar(self, p, trials, seed, stream=None):
        return bfc_espar(self.h, p, trials, seed, stream)

    def clrspar(self, colors, trials, seed, stream=None):
        return bfc_clrspar(self.h, colors, trials, seed, stream)

    def vsamp(self, k, trials, seed, proposal=None, want_draws=False, stream=None):
        return bfc_vsamp(self.h, k, trials, seed, proposal, want_draws, stream)

    def esamp(self, k, trials, seed, reps=0, want_draws=False, stream=None):
        return bfc_esamp(self.h, k, reps, trials, seed, want_draws, stream)

    def wsamp(self, k, trials, seed, want_draws=False, stream=None):
        return bfc_wsamp(self.h, k, trials, seed, want_draws, stream)

    def close(self):
        if self.h:
            bfc_graph_free(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
