"""Pins of the oracle's fast mode (the paper's resized and resampled
sequences): coordinates scaled to a coarser frame, a random share of the
events kept.

The scaling is checked against integer closed forms and the frame clamp, the
sampling against SplitMix64 as synth/rng.py computes it (an independent
implementation of the same published generator) and against its binomial
spread, and the coarse windows against known-D recovery.
"""
import math

import numpy as np
import pytest

import oracle as O
from synth import make_window
from synth.rng import splitmix64


def window(W, H, foe, x, y, t, tau=0.5):
    return O.Window(W, H, foe[0], foe[1], np.asarray(x, np.int16), np.asarray(y, np.int16),
                    np.asarray(t, np.float32), 0.0, tau)


def test_identity_when_nothing_changes(oracle_lib):
    rng = np.random.default_rng(1)
    w = window(50, 40, (25.0, 20.0), rng.integers(0, 50, 300), rng.integers(0, 40, 300),
               rng.random(300).astype(np.float32) * 0.5)
    r = O.resample(w, 50, 40, 1.0, 7)
    assert np.array_equal(r.x, w.x) and np.array_equal(r.y, w.y) and np.array_equal(r.t, w.t)
    assert (r.c.foe_x, r.c.foe_y) == (25.0, 20.0)


def test_half_resolution_is_nearest_coarse_pixel(oracle_lib):
    # k = 1/2 exactly: x2 = floor(x/2 + 1/2) = (x + 1) // 2, clamped to W2 - 1.
    x = np.arange(64)
    y = np.arange(64) % 48
    w = window(64, 48, (31.5, 23.0), x, y, np.zeros(64, np.float32))
    r = O.resample(w, 32, 24, 1.0, 3)
    assert np.array_equal(r.x, np.minimum((x + 1) // 2, 31))
    assert np.array_equal(r.y, np.minimum((y + 1) // 2, 23))
    assert (r.c.foe_x, r.c.foe_y) == (15.75, 11.5)


def test_the_foe_maps_like_a_frame_point(oracle_lib):
    # An anisotropic resize (640x480 -> 160x240: a quarter of the columns,
    # half the rows): an event on an integer FOE lands in the coarse pixel
    # nearest the coarse FOE, on each axis separately, so that the radial
    # geometry of Eq. (11) carries over to the coarse frame.
    for fx, fy in ((320.0, 240.0), (100.0, 400.0), (600.0, 30.0)):
        w = window(640, 480, (fx, fy), [int(fx)], [int(fy)], [0.25])
        r = O.resample(w, 160, 240, 1.0, 0)
        assert abs(r.c.foe_x - r.x[0]) <= 0.5 and abs(r.c.foe_y - r.y[0]) <= 0.5, (fx, fy)
        assert (r.c.foe_x, r.c.foe_y) == (fx / 4.0, fy / 2.0)


def test_clamp_at_the_far_edge(oracle_lib):
    # W = 5 -> W2 = 2: k = 0.4 (binary32); x = 4 maps to floor(2.1) = 2, clamped to 1.
    w = window(5, 5, (2.0, 2.0), [0, 1, 2, 3, 4], [4, 3, 2, 1, 0], np.zeros(5, np.float32))
    r = O.resample(w, 2, 2, 1.0, 0)
    want = [math.floor(float(np.float32(v) * np.float32(np.float32(2) / np.float32(5))) + 0.5) for v in range(5)]
    assert list(r.x) == [min(v, 1) for v in want]


def test_sampling_matches_splitmix64(oracle_lib):
    n, keep, seed = 5000, 0.25, 12345
    rng = np.random.default_rng(2)
    w = window(64, 64, (32.0, 32.0), rng.integers(0, 64, n), rng.integers(0, 64, n),
               (rng.random(n) * 0.5).astype(np.float32))
    r = O.resample(w, 64, 64, keep, seed)
    key = splitmix64(np.uint64(seed), np.uint64(0))
    top = splitmix64(key, np.arange(n, dtype=np.uint64)) >> np.uint64(40)
    kept = top < np.uint64(math.floor(keep * 2 ** 24))
    assert np.array_equal(r.t, w.t[kept]) and np.array_equal(r.x, w.x[kept])


def test_kept_share_is_binomial(oracle_lib):
    n, keep = 200_000, 0.25
    w = window(10, 10, (5.0, 5.0), np.zeros(n), np.zeros(n), np.zeros(n, np.float32))
    m = O.resample(w, 10, 10, keep, 99).x.size
    assert abs(m - n * keep) <= 4 * math.sqrt(n * keep * (1 - keep))
    assert O.resample(w, 10, 10, 0.0, 99).x.size == 0


def test_coarse_window_recovers_known_D(oracle_lib):
    # 640x480 at D = 0.35 scaled to 160x120 with a quarter of the events: one
    # coarse pixel at a typical radius of 60-100 coarse pixels spans
    # 1/(r tau) ~ 0.04 in D, so the estimate lands within 0.05.
    w = make_window(640, 480, 320.0, 240.0, 28000, 800, 12000, 0.35, 0.3, 2000)
    win = O.resample(O.Window.of(w), 160, 120, 0.25, 5)
    assert 8000 < win.x.size < 12000
    r = O.solve(win, -1.0, 1.0, 1e-4, 0.0, 16)
    assert abs(r["D_star"] - 0.35) <= 0.05
