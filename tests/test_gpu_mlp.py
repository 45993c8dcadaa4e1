"""The learned-proposal network on the GPU against the fp64 oracle, and what it gains.

Features, bf16 rounding, forward and gradient are compared with oracle.mlp;
training is checked to reduce the loss; the trained proposal is checked to be
unbiased and to shrink VSamp's exact single-draw variance on a held-out graph.
"""
import math

import numpy as np
import pytest

from oracle import mlp as M
from paper_1801_00338_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def bfc():
    import torch
    assert torch.cuda.is_available()
    from paper_1801_00338_gb300 import build as B
    B.build()
    from paper_1801_00338_gb300 import bfc as mod
    mod.load()
    return mod


@pytest.fixture(scope="module")
def small():
    return synth.chung_lu_scaled(3000, 9000, 40_000, 2.1, 2.4, 5)


def _bf16_values(wb):
    """bfloat16 bits (int16 tensor) -> float64 numpy."""
    import torch
    return wb.view(torch.bfloat16).to(torch.float64).cpu().numpy()


def test_features_match_oracle(bfc, small):
    g = small
    with bfc.Graph(g.u, g.v, g.nU, g.nV) as G:
        f = bfc.bfc_features(G.h, g.nU + g.nV).cpu().numpy()
    want = M.features(g.u, g.v, g.nU, g.nV)
    assert np.allclose(f, want, rtol=2e-6, atol=2e-7)


def test_bf16_copy_matches_oracle_rounding(bfc):
    import torch
    w = np.random.default_rng(3).normal(0, 0.4, bfc.MLP_PARAMS).astype(np.float32)
    wb = bfc.bfc_mlp_to_bf16(torch.from_numpy(w).cuda())
    assert np.array_equal(_bf16_values(wb), M.bf16(w))


def test_forward_within_1e3_of_fp64(bfc, small):
    import torch
    g = small
    w = np.random.default_rng(4).normal(0, 0.3, bfc.MLP_PARAMS).astype(np.float32)
    wb = bfc.bfc_mlp_to_bf16(torch.from_numpy(w).cuda())
    with bfc.Graph(g.u, g.v, g.nU, g.nV) as G:
        X = bfc.bfc_features(G.h, g.nU + g.nV)
    y = bfc.bfc_mlp_forward(wb, X).cpu().numpy().astype(np.float64)
    want = M.forward(M.bf16(w), X.cpu().numpy().astype(np.float64))
    rel = np.abs(y - want) / np.maximum(np.abs(want), 1.0)
    assert rel.max() <= 1e-3


def test_gradient_matches_fp64(bfc, small):
    import torch
    g = small
    rng = np.random.default_rng(6)
    w = rng.normal(0, 0.3, bfc.MLP_PARAMS).astype(np.float32)
    wb = bfc.bfc_mlp_to_bf16(torch.from_numpy(w).cuda())
    with bfc.Graph(g.u, g.v, g.nU, g.nV) as G:
        X = bfc.bfc_features(G.h, g.nU + g.nV)
        bU, bV, _ = G.per_vertex()
        T = bfc.bfc_mlp_targets(torch.cat([bU, bV]))
    idx = rng.integers(0, g.nU + g.nV, 1500).astype(np.int32)  # 12 tiles, ragged last
    grad, loss = bfc.bfc_mlp_grad(wb, X, T, torch.from_numpy(idx).cuda())
    Xh = X.cpu().numpy().astype(np.float64)[idx]
    Th = T.cpu().numpy().astype(np.float64)[idx]
    want_loss, want = M.loss_and_grad(M.bf16(w), Xh, Th)
    got = grad.cpu().numpy().astype(np.float64)
    assert float(loss.item()) == pytest.approx(want_loss, rel=1e-4)
    scale = np.abs(want).max()
    assert np.abs(got - want).max() <= 1e-4 * scale


def _weight_tolerance(w_orc):
    """Per-weight bound between the kernel's float32 exp(s - max s) 2^24 and the
    oracle's float64 one: s - max s rounds once in float32 (relative 2^-24, which
    moves 2^24 e^d by at most |d| e^d <= 1/e units), expf is within 2 ulp
    (relative 2^-22, at most 4 units at 2^24), and the two floors can differ by 1.
    The exp term is doubled for margin."""
    return 2.0 + w_orc.astype(np.float64) * 2.0 ** -21


def test_proposal_weights_match_oracle_score_weights(bfc):
    """bfc_proposal_from_scores's integer weights, element by element, against
    oracle.mlp.score_weights on scores spanning the clamp at 1, the full unit and
    ties at the maximum; the stored sum W is the sum of the weights."""
    import torch
    rng = np.random.default_rng(11)
    nU, nV = 300, 500
    u, v = synth.uniform_bipartite(nU, nV, 2500, 3)
    n = nU + nV
    cases = [
        rng.normal(0.0, 3.0, n),                          # wide spread, many clamped to 1
        rng.uniform(-0.5, 0.5, n),                        # all within the full unit
        np.where(rng.random(n) < 0.1, 4.0, rng.normal(0.0, 1.0, n)),  # ties at the maximum
        np.full(n, -7.25),                                # all equal
    ]
    with bfc.Graph(u, v, nU, nV) as G:
        for s64 in cases:
            s32 = s64.astype(np.float32)
            prop = bfc.bfc_proposal_from_scores(G.h, torch.from_numpy(s32).cuda())
            try:
                w, W = bfc.bfc_proposal_weights(prop, n)
            finally:
                bfc.bfc_proposal_free(prop)
            want = M.score_weights(s32.astype(np.float64))
            diff = np.abs(w.astype(np.float64) - want.astype(np.float64))
            assert np.all(diff <= _weight_tolerance(want))
            assert W == int(w.astype(np.uint64).sum())
            assert w.min() >= 1 and w.max() == 1 << 24


def test_training_reduces_loss_and_proposal_gains(bfc):
    """Train on small generated graphs; on a held-out graph the learned mixture
    proposal keeps VSamp unbiased (exactly, by the importance weights) and its
    exact single-draw variance falls well below uniform VSamp's."""
    import torch
    from paper_1801_00338_gb300 import learned as Ln
    params = Ln.training_graph_params(12, 21, 5e3, 8e4)
    graphs = []
    for i, (nU, nV, m, gu, gv) in enumerate(params):
        u, v = synth.chung_lu_bipartite(nU, nV, m, gu, gv, 900 + i)
        graphs.append((u, v, nU, nV))
    data = Ln.dataset_from_graphs(graphs)
    tr = Ln.Trainer(seed=0, lr=3e-3, out_bias=float(data.T.mean().item()))
    before = tr.mse(data)
    tr.fit(data, steps=400, batch=16384)
    after = tr.mse(data)
    assert after < 0.5 * before
    # held-out graph
    h = synth.chung_lu_scaled(4000, 8000, 120_000, 2.3, 2.3, 777)
    with bfc.Graph(h.u, h.v, h.nU, h.nV) as G:
        bU, bV, B = G.per_vertex()
        b = np.concatenate([bU.cpu().numpy(), bV.cpu().numpy()]).astype(np.float64)
        s = Ln.scores(G, tr.wb).cpu().numpy()
        prop = bfc.bfc_proposal_from_scores(G.h, Ln.scores(G, tr.wb))
        try:
            k, trials = 64, 400
            est = G.vsamp(k, trials, 99, proposal=prop)
        finally:
            bfc.bfc_proposal_free(prop)
    w = M.score_weights(s).astype(np.float64)
    q = 0.5 / w.size + 0.5 * w / w.sum()
    var_u = Ln.single_draw_variance(b)
    var_l = Ln.single_draw_variance(b, q)
    assert var_l < 0.25 * var_u
    se = math.sqrt(var_l / k / trials)
    assert abs(np.mean(est) - B) <= 3 * se
