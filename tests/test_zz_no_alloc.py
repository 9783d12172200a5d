"""The allocation-free contrast entry point, checked against dd_contrast and
the oracle.

Some users of this library cannot allocate device memory while they
evaluate contrasts: flight software whose rules forbid allocation after
start-up, or a plugin running inside a host process that owns all device
memory through its own capped pool.  dd_contrast_noalloc serves them from
one fixed static device array instead of cudaMalloc.  It must return
exactly the keys dd_contrast returns (keys are exact integers, so the
tolerance is zero), also on a second call that finds the first call's data
still in the shared array, and the keys of Eqs. 11-13 as the oracle
computes them; after its first call on a device (which may load the
library's device code), further calls leave the device's free memory
unchanged.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
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


def oracle_keys(w, Ds):
    win = O.Window.of(w)
    return [O.contrast(win, float(D))[0] for D in Ds]


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
        assert got == oracle_keys(w, Ds)


def test_noalloc_leaves_free_device_memory_unchanged():
    w = window_config2()
    ev = dd.Events.of(w, device="cuda")
    Ds = np.linspace(-1.0, 1.0, 80).astype(np.float32)
    first = dd.dd_contrast_noalloc(w.W, w.H, w.foe_x, w.foe_y, ev, Ds)   # may load the device code
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    again = [dd.dd_contrast_noalloc(w.W, w.H, w.foe_x, w.foe_y, ev, Ds) for _ in range(3)]
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert all(k == first for k in again)


@pytest.mark.parametrize("W,H,fx,fy,seed", [(4096, 4096, 4096.0, 0.0, 77), (1, 4096, 0.0, 4096.0, 78),
                                            (4096, 1, 0.0, 1.0, 79)])
def test_noalloc_largest_and_degenerate_frames(W, H, fx, fy, seed):
    # The largest frame (683 row bands, 4096 sort bins) and one-pixel-wide or
    # -high frames, FOE on a corner, a few thousand events.
    w = make_window(W, H, fx, fy, 2000, 60, 500, 0.25, 0.3, seed)
    ev = dd.Events.of(w, device="cuda")
    Ds = np.array([0.0, 0.25, -0.7, 0.9, 1.5, -3.0], np.float32)
    got = dd.dd_contrast_noalloc(W, H, fx, fy, ev, Ds)
    assert got == reference_keys(w, ev, Ds)
    assert got == oracle_keys(w, Ds)


def test_noalloc_rejects_what_dd_contrast_rejects():
    # Rejected on the host before any GPU work: the pointers are never read.
    x = torch.zeros(1, dtype=torch.int16, device="cuda")
    t = torch.zeros(1, dtype=torch.float32, device="cuda")
    ev = dd.Events(x, x, t, 0.0, 0.3)
    ev.c.n = dd.DD_NOALLOC_MAX_EVENTS + 1
    with pytest.raises(dd.DDError) as e:
        dd.dd_contrast_noalloc(640, 480, 320.0, 240.0, ev, [0.1])
    assert e.value.status == dd.DD_ERR_CAPACITY
    ok = dd.Events(x, x, t, 0.0, 0.3)
    for D in (float("nan"), 2.6, -214.0):                # outside -64 <= D tau <= 3/4
        with pytest.raises(dd.DDError) as e:
            dd.dd_contrast_noalloc(640, 480, 320.0, 240.0, ok, [D])
        assert e.value.status == dd.DD_ERR_ARG
    bad = dd.Events(x, x, t, 0.0, 0.3)
    bad.c.tau = 0.0
    with pytest.raises(dd.DDError) as e:
        dd.dd_contrast_noalloc(640, 480, 320.0, 240.0, bad, [0.1])
    assert e.value.status == dd.DD_ERR_ARG
    assert ctypes.sizeof(dd.dd_i128) == 16
