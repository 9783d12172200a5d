"""The stream report's metrics (host arithmetic): 0.5 s averaging and the
divergence error in percent, on hand-made values."""
import numpy as np

from paper_2209_13168_gb300.stream import divergence_error_pct, resolution_average


def test_resolution_average_bins_by_time():
    t = np.array([0.2, 0.3, 0.4, 0.5, 0.6, 1.2])
    v = np.array([1.0, 2.0, 3.0, 10.0, 20.0, 5.0])
    tb, vb = resolution_average(t, v, 0.5)
    assert np.allclose(tb, [0.3, 0.55, 1.2]) and np.allclose(vb, [2.0, 15.0, 5.0])


def test_divergence_error_against_the_descent():
    # truth at t: 1/(20 - t); an estimate 10% high is a 10% error
    t = np.array([0.0, 10.0, 19.0])
    D = 1.1 / (20.0 - t)
    assert np.allclose(divergence_error_pct(D, t), 10.0)
    assert divergence_error_pct([0.05], [0.0])[0] == 0.0
