"""The seeded input generator (shared by both sides; no reconstructor arithmetic)."""
import numpy as np

from paper_1806_07938_gb300 import workloads as W


def small():
    return dict(W.config("lgs_mid"), n=8, D=8 * 39.0 / 74)


def test_sequence_step0_is_the_frame_and_noise_is_fresh():
    cfg = small()
    grids = W._grids(cfg)
    seq, sig = W.slope_sequence(cfg, 2, 3, seed=4, dt=0.0)
    _, sig_f = W.slope_frames(cfg, 1, seed=4)
    assert np.array_equal(sig, sig_f)
    for j in range(2):
        clean = W._clean_frame(cfg, 4, j, 512, grids)
        for t in range(3):
            # dt = 0: every step sees the same screens; only the noise differs
            resid = (seq[t, j] - clean) / sig[:, None, None, None]
            assert abs(resid.std() - 1.0) < 0.15
        assert not np.array_equal(seq[0, j], seq[1, j])


def test_sequence_frozen_flow_moves_the_screens():
    cfg = small()
    a, _ = W.slope_sequence(cfg, 1, 2, seed=4, dt=1e-3)
    b, _ = W.slope_sequence(cfg, 1, 2, seed=4, dt=0.05)
    d_small = np.std(a[1] - a[0])
    d_large = np.std(b[1] - b[0])
    assert d_large > 2 * d_small          # 50 ms of wind decorrelates far more than 1 ms
    c, _ = W.slope_sequence(cfg, 1, 2, seed=4, dt=1e-3)
    assert np.array_equal(a, c)           # deterministic
