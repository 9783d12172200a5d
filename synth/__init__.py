"""Seeded synthetic event windows shared by the tests, the benchmark and smoke().

This package holds only input generation (a counter-based random stream and a
scene model of a camera descending onto a fronto-parallel plane).  It contains
none of the estimator's arithmetic: no warp, no image of warped events, no
contrast and no bound.
"""
from .rng import splitmix64, uniform01, stream_key
from .descent import Window, make_window, window_config1, window_config2, batch_config3, serve_config5

__all__ = [
    "splitmix64", "uniform01", "stream_key", "Window", "make_window",
    "window_config1", "window_config2", "batch_config3", "serve_config5",
]
