"""The allocation-free contrast entry point, checked against dd_contrast.

Some users of this library cannot allocate device memory while they
evaluate contrasts: flight software whose rules forbid allocation after
start-up, or a plugin running inside a host process that owns all device
memory through its own capped pool.  dd_contrast_noalloc serves them from
one fixed static device array instead of cudaMalloc.  It must return
exactly the keys dd_contrast returns (keys are exact integers, so the
tolerance is zero), also on a second call that finds the first call's data
still in the shared array.
"""
import ctypes

import numpy as np
import pytest

from synth import make_window, window_config2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2209_13168_gb300 as dd  # noqa: E402


def reference_keys(w, ev, Ds):
    ctx = dd.Context(w.W, w.H, w.foe_x, w.foe_y)
    try:
        return ctx.contrast(ev, Ds)[0]
    finally:
        ctx.close()


def test_noalloc_matches_dd_contrast_on_two_calls_in_a_row():
    # First a large window, then a smaller one with another frame size, so the
    # second call runs over what the first left in the static array.
    big = window_config2()
    small = make_window(346, 260, 173.0, 130.0, 3000, 150, 1000, 0.2, 0.5, seed=1000)
    rng = np.random.default_rng(12)
    calls = []
    for w in (big, small):
        ev = dd.Events.of(w, device="cuda")
        Ds = np.concatenate([[0.0, w.D_true], rng.uniform(-1.0, 1.0, 70)]).astype(np.float32)
        calls.append((w, ev, Ds, dd.dd_contrast_noalloc(w.W, w.H, w.foe_x, w.foe_y, ev, Ds)))
    for w, ev, Ds, got in calls:
        assert got == reference_keys(w, ev, Ds)


def test_noalloc_rejects_windows_beyond_its_capacity():
    # Rejected on the host before any GPU work: the pointers are never read.
    x = torch.zeros(1, dtype=torch.int16, device="cuda")
    t = torch.zeros(1, dtype=torch.float32, device="cuda")
    ev = dd.Events(x, x, t, 0.0, 0.3)
    ev.c.n = dd.DD_NOALLOC_MAX_EVENTS + 1
    with pytest.raises(dd.DDError) as e:
        dd.dd_contrast_noalloc(640, 480, 320.0, 240.0, ev, [0.1])
    assert e.value.status == dd.DD_ERR_CAPACITY
    assert ctypes.sizeof(dd.dd_i128) == 16
