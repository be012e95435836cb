"""Pins of the seeded input generators that stand in for the paper's data."""
import numpy as np


def test_paper2d_generators():
    """The inputs standing in for the paper's 2D experiments (Sec. 4.2):
    300 x 400 x 3, 5 x 5 kernels summing to one per channel, the motion kernel
    on the main diagonal, noise of standard deviation 0.02, and for the
    semi-blind case a generating kernel that is the motion kernel blurred
    further (not the known one)."""
    from paper_2502_09758_gb300 import synth
    m = synth.paper2d_motion(0)
    s = synth.paper2d_semiblind(0)
    for inst in (m, s):
        assert inst.shape == (3, 300, 400) and inst.K == 5
        np.testing.assert_allclose(inst.b_true.sum(axis=(1, 2)), 1.0, atol=1e-12)
        np.testing.assert_allclose(inst.a.sum(axis=(1, 2)), 1.0, atol=1e-12)
        resid = inst.y - synth._periodic_blur(inst.b_true, inst.x_true)
        assert abs(resid.std() - 0.02) < 5e-4
    np.testing.assert_array_equal(m.a[0], np.eye(5) / 5)
    np.testing.assert_array_equal(s.a[0], np.eye(5) / 5)
    assert np.abs(s.b_true[0] - np.eye(5) / 5).max() > 0.02      # the unknown extra blur
    assert np.allclose(s.b_true[0], s.b_true[0].T)               # diagonal motion and Gaussian: symmetric
    assert synth.paper2d_motion(0).y.tobytes() == m.y.tobytes()  # seeded
