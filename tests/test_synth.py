"""The input generator is deterministic per seed and has the stated statistics."""
import numpy as np

import synth


def test_generators_are_seeded():
    a = synth.config_pair("plain_320x240")
    b = synth.config_pair("plain_320x240")
    assert np.array_equal(a.left, b.left) and np.array_equal(a.right, b.right)
    c = synth.config_pair("plain_320x240", seed=1)
    assert not np.array_equal(a.left, c.left)


def test_g1_statistics():
    p = synth.g1_pair(320, 240, 0)
    assert p.left.dtype == np.uint8 and p.left.shape == (240, 320)
    assert 110 < p.left.mean() < 146 and 30 < p.left.std() < 60
    assert 4.0 <= p.disp_right.min() and p.disp_right.max() <= 24.0 + 1e-9


def test_g2_statistics():
    p = synth.g2_pair(640, 480, 0)
    assert abs(p.disp_right.min() - 5) < 1e-9 and abs(p.disp_right.max() - 60) < 1e-9
    assert (p.left == 255).mean() > 0.005        # specular discs
    # the right view is the left warped by the ground truth (left grid)
    gt = p.gt_left()
    assert gt.min() >= 5 - 1e-6 and gt.max() <= 60 + 1e-6


def test_shift_pair_is_exact_shift():
    p = synth.shift_pair(64, 16, 0, 5)
    assert np.array_equal(p.left[:, 5:], p.right[:, :-5])
