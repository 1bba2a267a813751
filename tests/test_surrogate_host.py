"""Host-side pieces of the covariance surrogate (no GPU): the shipped weights, the seeded initial
weights, the trajectory error and the frame chunking of the training/evaluation module."""
import numpy as np

from oracle import surrogate as sgo
from paper_2403_12550_b300 import surrogate as S


def test_shipped_weights_load_and_are_finite():
    w = S.load_weights()
    assert w.shape == (S.N_WEIGHTS,) == (sgo.N_WEIGHTS,) and w.dtype == np.float32
    assert np.all(np.isfinite(w)) and np.abs(w).max() < 1e3
    # every layer is used (no all-zero layer)
    for part in sgo.split_weights(w):
        assert np.abs(part).max() > 0


def test_init_weights_seeded_he_normal():
    a, b = S.init_weights(3), S.init_weights(3)
    np.testing.assert_array_equal(a, b)
    assert not np.array_equal(a, S.init_weights(4))
    W1, W2, W3 = sgo.split_weights(a)
    for Wl, fan_in in ((W1, 75), (W2, 800), (W3, 800)):
        assert abs(Wl.std() - np.sqrt(2.0 / fan_in)) < 0.15 * np.sqrt(2.0 / fan_in)


def test_ate_rmse_and_chunks():
    gt = [np.eye(4) for _ in range(4)]
    est = [np.eye(4) for _ in range(4)]
    est[1][:3, 3] = [0.03, 0.0, 0.04]  # 5 cm off in one of four frames
    assert abs(S.ate_rmse(est, gt) - np.sqrt(0.05 ** 2 / 4)) < 1e-15
    ch = S._chunks(10, 3)
    assert sum(ch, []) == list(range(10)) and len(ch) == 3
