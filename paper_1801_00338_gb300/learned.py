"""The learned VSamp proposal: training on exact per-vertex counts and use.

An extension, not in the paper.  Algorithm 4 (VSamp) draws vertices
uniformly and returns b_v * n / 4; Lemma 4 shows the estimate is unbiased but
its variance grows with the spread of b_v.  Drawing v with probability q(v)
and returning b_v / (4 q(v)) is unbiased for any q > 0 and has zero variance
when q is proportional to b_v.  Here q mixes half uniform with half
proportional to exp(s_v), where s_v is a small network's guess of log1p(b_v)
from six cheap features; the uniform half keeps q >= 1/(2n), so the weights
stay bounded and the estimator unbiased whatever the network predicts.

Every numeric step runs in libbfc.so (features, forward, gradient, Adam,
proposal weights, sampling); this module only orchestrates: it draws the
training graphs, forms mini-batches and records timings.
"""
from __future__ import annotations

import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import bfc, synth

F, H = bfc.MLP_FEATURES, 64


# parameter vector offsets: W1[6][64], b1[64], W2[64][64], b2[64], W3[64], b3
OFF_W1, OFF_B1 = 0, F * H
OFF_W2 = OFF_B1 + H
OFF_B2 = OFF_W2 + H * H
OFF_W3 = OFF_B2 + H
OFF_B3 = OFF_W3 + H


def init_params(seed: int, out_bias: float = 0.0) -> np.ndarray:
    """Uniform Glorot initialisation of the weight matrices; zero hidden biases;
    the output bias starts at `out_bias` (e.g. the mean target)."""
    rng = np.random.default_rng(seed)
    p = np.zeros(bfc.MLP_PARAMS, np.float32)
    p[OFF_W1:OFF_B1] = rng.uniform(-1, 1, F * H) * math.sqrt(6.0 / (F + H))
    p[OFF_W2:OFF_B2] = rng.uniform(-1, 1, H * H) * math.sqrt(6.0 / (H + H))
    p[OFF_W3:OFF_B3] = rng.uniform(-1, 1, H) * math.sqrt(6.0 / (H + 1))
    p[OFF_B3] = out_bias
    return p


def training_graph_params(count: int, seed: int, m_lo: float, m_hi: float):
    """(nU, nV, m, gamma_u, gamma_v) per training graph: m log-uniform in
    [m_lo, m_hi], exponents uniform in [1.9, 2.8], |V| = 2 |U|, mean degree 20 on U."""
    r = synth.uniform01(seed, 0, 3 * count).reshape(count, 3)
    out = []
    for i in range(count):
        m = int(round(math.exp(math.log(m_lo) + r[i, 0] * (math.log(m_hi) - math.log(m_lo)))))
        nU = max(50, m // 20)
        nV = 2 * nU
        out.append((nU, nV, m, 1.9 + 0.9 * r[i, 1], 1.9 + 0.9 * r[i, 2]))
    return out


@dataclass
class Dataset:
    X: object = None      # torch float32 [n, 6] on the device
    T: object = None      # torch float32 [n]
    sizes: list = field(default_factory=list)


def dataset_from_graphs(graphs) -> Dataset:
    """Features and log1p(b) targets of every vertex of every graph (exact b from vBFC)."""
    import torch
    Xs, Ts, sizes = [], [], []
    for u, v, nU, nV in graphs:
        with bfc.Graph(u, v, nU, nV) as G:
            X = bfc.bfc_features(G.h, nU + nV)
            bU, bV, _ = G.per_vertex()
            T = bfc.bfc_mlp_targets(torch.cat([bU, bV]))
        Xs.append(X)
        Ts.append(T)
        sizes.append(nU + nV)
    return Dataset(torch.cat(Xs), torch.cat(Ts), sizes)


def save_checkpoint(path: str, state: dict):
    """Write a training state (see Trainer.state) to an .npz file: the fp32
    master weights, both Adam moments, the step count, the learning rate, the
    mini-batch generator's state and any extra arrays (e.g. the training
    graphs' parameters), so that training resumes exactly where it stopped."""
    import json
    arrays = {k: np.asarray(v) for k, v in state.items() if k != "rng"}
    arrays["rng_json"] = np.array(json.dumps(state.get("rng")))
    np.savez(path, **arrays)


def load_checkpoint(path: str) -> dict:
    import json
    with np.load(path, allow_pickle=False) as z:
        st = {k: z[k] for k in z.files if k != "rng_json"}
        st["rng"] = json.loads(str(z["rng_json"]))
    st["step"] = int(st["step"])
    st["lr"] = float(st["lr"])
    return st


def rng_from_state(state) -> np.random.Generator:
    """A PCG64 generator positioned at a saved bit-generator state."""
    rng = np.random.default_rng()
    rng.bit_generator.state = state
    return rng


class Trainer:
    """Adam on the fp32 master weights; the bf16 copy feeds the kernels."""

    def __init__(self, seed: int = 0, lr: float = 1e-3, out_bias: float = 0.0):
        import torch
        self.w = torch.from_numpy(init_params(seed, out_bias)).cuda()
        self.wb = bfc.bfc_mlp_to_bf16(self.w)
        self.m = torch.zeros_like(self.w)
        self.v = torch.zeros_like(self.w)
        self.lr = lr
        self.step = 0
        self.history = []
        self.rng = None  # mini-batch generator, seeded by the first fit()

    def state(self, **extra) -> dict:
        """The training state as host arrays (for save_checkpoint)."""
        st = {"w": self.w.cpu().numpy(), "m": self.m.cpu().numpy(), "v": self.v.cpu().numpy(), "step": self.step,
              "lr": self.lr, "rng": self.rng.bit_generator.state if self.rng is not None else None}
        st.update(extra)
        return st

    def load_state(self, st: dict):
        """Resume from a state written by save_checkpoint: weights, Adam
        moments, step count and the mini-batch generator's position."""
        import torch
        self.w = torch.from_numpy(np.asarray(st["w"], np.float32)).cuda()
        self.m = torch.from_numpy(np.asarray(st["m"], np.float32)).cuda()
        self.v = torch.from_numpy(np.asarray(st["v"], np.float32)).cuda()
        self.wb = bfc.bfc_mlp_to_bf16(self.w)
        self.step = int(st["step"])
        self.lr = float(st["lr"])
        self.rng = rng_from_state(st["rng"]) if st.get("rng") is not None else None

    def fit(self, data: Dataset, steps: int, batch: int = 65536, seed: int = 1, log_every: int = 50):
        import torch
        n = data.X.shape[0]
        if self.rng is None:
            self.rng = np.random.default_rng(seed)
        rng = self.rng
        for s in range(steps):
            idx = torch.from_numpy(rng.integers(0, n, min(batch, n), dtype=np.int64).astype(np.int32)).cuda()
            grad, loss = bfc.bfc_mlp_grad(self.wb, data.X, data.T, idx)
            self.step += 1
            bfc.bfc_mlp_adam(self.w, self.wb, self.m, self.v, grad, self.lr, self.step)
            if s % log_every == 0 or s == steps - 1:
                self.history.append((self.step, float(loss.item())))
        return self.history

    def mse(self, data: Dataset) -> float:
        y = bfc.bfc_mlp_forward(self.wb, data.X)
        return float(((y - data.T) ** 2).mean().item())


def scores(G: "bfc.Graph", wb):
    """Network scores of every vertex of G (U first)."""
    X = bfc.bfc_features(G.h, G.nU + G.nV)
    return bfc.bfc_mlp_forward(wb, X)


def proposal(G: "bfc.Graph", wb) -> int:
    """A bfc_vsamp proposal handle built from the network's scores."""
    return bfc.bfc_proposal_from_scores(G.h, scores(G, wb))


def mixture_q(prop: int, n: int) -> np.ndarray:
    """q of bfc_vsamp's mixture for a proposal handle, from the integer weights
    the library stores: q(i) = 1/(2n) + w_i / (2W) (float64 on the host)."""
    w, W = bfc.bfc_proposal_weights(prop, n)
    return 0.5 / n + 0.5 * w.astype(np.float64) / float(W)


def single_draw_variance(b: np.ndarray, q: np.ndarray | None = None) -> float:
    """Exact variance of one draw b_v / (4 q(v)): sum_v b_v^2 / (16 q(v)) - B^2."""
    b = np.asarray(b, dtype=np.float64)
    if q is None:
        q = np.full(b.size, 1.0 / b.size)
    B = b.sum() / 4.0
    return float(np.sum(b * b / (16.0 * q)) - B * B)


def draws_for_median_error(var1: float, B: float, rel: float = 0.01) -> int:
    """Draws k at which the median |estimate - B| / B of a k-draw mean is `rel`
    (normal approximation: median |N(0, s^2)| = 0.6745 s)."""
    return max(1, int(math.ceil((0.6744897501960817 / rel) ** 2 * var1 / (B * B))))


def _train_graph_job(args):
    i, (nU, nV, m, gu, gv), seed = args
    u, v = synth.chung_lu_bipartite(nU, nV, m, gu, gv, seed)
    return u, v, nU, nV


def train_proposal(count: int = 200, m_lo: float = 1e5, m_hi: float = 2e7, steps: int = 2000, seed: int = 0,
                   workers: int = 0):
    """Train the proposal network: `count` Chung-Lu graphs with m log-uniform in
    [m_lo, m_hi] and exponents uniform in [1.9, 2.8] (generated by spawned
    worker processes), exact per-vertex labels from the library, `steps` Adam
    steps of 65,536 rows.  Returns (trainer, info)."""
    import multiprocessing as mp
    import os
    import torch
    info = {"train_graphs": count, "train_m_range": [m_lo, m_hi], "steps": steps}
    t0 = time.perf_counter()
    params = training_graph_params(count, seed + 21, m_lo, m_hi)
    jobs = [(i, prm, 10_000 + seed * 1000 + i) for i, prm in enumerate(params)]
    workers = workers or min(16, os.cpu_count() or 1)
    with mp.get_context("spawn").Pool(workers) as pool:
        graphs = pool.map(_train_graph_job, jobs, chunksize=2)
    info["train_edges"] = int(sum(len(g[0]) for g in graphs))
    info["gen_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    data = dataset_from_graphs(graphs)
    del graphs
    torch.cuda.synchronize()
    info["label_s"] = time.perf_counter() - t0
    tr = Trainer(seed=seed, lr=3e-3, out_bias=float(data.T.mean().item()))
    info["mse_before"] = tr.mse(data)
    t0 = time.perf_counter()
    tr.fit(data, steps=steps, batch=65536)
    torch.cuda.synchronize()
    info["train_s"] = time.perf_counter() - t0
    info["mse_after"] = tr.mse(data)
    return tr, info


def equal_time(G: "bfc.Graph", b: np.ndarray, B: int, wb, trials: int = 3, seed: int = 0, rel: float = 0.01) -> dict:
    """Uniform against learned VSamp (Algorithm 4; the learned mixture reweighted
    by Horvitz-Thompson) at equal GPU time on one graph: the learned arm runs
    the draws its exact variance predicts for a `rel` median error, its time
    including the proposal build (features, network, weights, prefix table);
    the uniform arm then gets the same time per trial.  Both arms' median
    relative errors over `trials` trials are measured."""
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    prop = proposal(G, wb)
    torch.cuda.synchronize()
    t_prop = time.perf_counter() - t0
    try:
        n = G.nU + G.nV
        q = mixture_q(prop, n)
        var_u = single_draw_variance(b)
        var_l = single_draw_variance(b, q)
        k_l = draws_for_median_error(var_l, B, rel)
        k_u_pred = draws_for_median_error(var_u, B, rel)
        G.vsamp(1024, 2, seed + 99, proposal=prop)  # warm-up of both sides' layouts
        G.vsamp(1024, 2, seed + 98)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        est_l = G.vsamp(k_l, trials, seed + 1, proposal=prop)
        torch.cuda.synchronize()
        t_l = (time.perf_counter() - t0) / trials + t_prop
        # uniform: a call's fixed cost and per-draw time from two pilots, then
        # the draws that fill t_l
        pilot = []
        for kp in (1 << 20, 1 << 22):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            G.vsamp(kp, 1, seed + 2)
            torch.cuda.synchronize()
            pilot.append((kp, time.perf_counter() - t0))
        t_draw_u = max((pilot[1][1] - pilot[0][1]) / (pilot[1][0] - pilot[0][0]), 1e-12)
        t_fixed = max(0.0, pilot[0][1] - pilot[0][0] * t_draw_u)
        k_u = max(1, int((t_l - t_fixed) / t_draw_u))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        est_u = G.vsamp(k_u, trials, seed + 3)
        torch.cuda.synchronize()
        t_u = (time.perf_counter() - t0) / trials
    finally:
        bfc.bfc_proposal_free(prop)
    err_l = np.abs(np.asarray(est_l, np.float64) - B) / B
    err_u = np.abs(np.asarray(est_u, np.float64) - B) / B
    # the median relative error the exact single-draw variance predicts (normal
    # approximation: the median of |N(0, 1)| is 0.6745)
    pred = lambda var1, k: 0.6744897501960817 * math.sqrt(var1 / k) / B
    return {"trials": trials, "target_rel_err": rel,
            "learned": {"draws": int(k_l), "s_per_trial": t_l, "proposal_build_s": t_prop,
                        "median_rel_err": float(np.median(err_l)), "predicted_median_rel_err": pred(var_l, k_l),
                        "var_single_draw": var_l},
            "uniform": {"draws": int(k_u), "s_per_trial": t_u, "median_rel_err": float(np.median(err_u)),
                        "predicted_median_rel_err": pred(var_u, k_u), "var_single_draw": var_u,
                        "draws_for_target": int(k_u_pred), "s_for_target": k_u_pred * t_draw_u},
            "time_ratio_to_target": t_l / (k_u_pred * t_draw_u),
            "error_ratio_at_equal_time": float(np.median(err_l) / max(np.median(err_u), 1e-300))}
