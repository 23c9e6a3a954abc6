"""The seeded input generators: determinism, shapes, ranges, planted MVs."""
import numpy as np

from paper_2508_05990_b300 import synth


def test_planted_pair_deterministic_and_12bit():
    a = synth.planted_pair(1000)
    b = synth.planted_pair(1000)
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)
    f0, f1, mv = a
    assert f0.dtype == np.uint16 and f0.shape == (256, 256) and f0.max() <= 4095
    assert f1.max() <= 4095
    assert mv.shape == (16, 16, 2) and (mv % 2 == 0).all() and np.abs(mv).max() <= 8


def test_pan_clip_shapes():
    c = synth.pan_clip(3, 64, 96, n_frames=3, rect_size=(8, 24))
    assert c.shape == (3, 64, 96) and c.dtype == np.uint16 and c.max() <= 4095
    np.testing.assert_array_equal(c, synth.pan_clip(3, 64, 96, n_frames=3, rect_size=(8, 24)))


def test_features_layouts():
    a = synth.features(1, 4, 5, 6, n=2)
    b = synth.features(1, 4, 5, 6, n=2, layout="NHWC")
    assert a.shape == (2, 4, 5, 6) and b.shape == (2, 5, 6, 4) and a.dtype == np.float32


def test_round_half_away():
    np.testing.assert_array_equal(synth.round_clip(np.array([0.5, 1.5, 2.49, -0.5, 4095.6])),
                                  np.array([1, 2, 2, 0, 4095], np.uint16))
