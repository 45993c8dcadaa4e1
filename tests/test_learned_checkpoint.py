"""Checkpoint and resume of the learned proposal's training (host logic, no GPU)."""
import numpy as np


def test_training_checkpoint_round_trip(tmp_path):
    """The learned proposal's training state (fp32 weights, Adam moments, step,
    learning rate, mini-batch generator) survives a save and load, and the
    restored generator continues the same batch sequence (host logic only)."""
    from paper_1801_00338_gb300 import learned as Lrn
    rng = np.random.default_rng(1)
    P = 4673
    w, m, v = (rng.standard_normal(P).astype(np.float32) for _ in range(3))
    gen = np.random.default_rng(77)
    gen.integers(0, 1000, 50)                      # some batches already drawn
    st = {"w": w, "m": m, "v": v, "step": 123, "lr": 3e-3, "rng": gen.bit_generator.state,
          "train_params": np.arange(10, dtype=np.float64)}
    path = str(tmp_path / "ckpt.npz")
    Lrn.save_checkpoint(path, st)
    back = Lrn.load_checkpoint(path)
    for k in ("w", "m", "v", "train_params"):
        assert np.array_equal(back[k], st[k]) and back[k].dtype == st[k].dtype
    assert back["step"] == 123 and back["lr"] == 3e-3
    resumed = Lrn.rng_from_state(back["rng"])
    assert np.array_equal(resumed.integers(0, 1000, 64), gen.integers(0, 1000, 64))
