"""The fast mode (resized and resampled windows) on the GPU against the oracle:
the coarse window event for event and in order, and the exact solve on it."""
import numpy as np
import pytest

import oracle as O
from synth import make_window, window_config1, window_config2, serve_config5

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2209_13168_gb300 as dd  # noqa: E402


def check(w, W2, H2, keep, seed):
    win = O.Window.of(w)
    want = O.resample(win, W2, H2, keep, seed)
    fx, fy = dd.dd_resample_foe(w.W, w.H, w.foe_x, w.foe_y, W2, H2)
    assert (fx, fy) == (want.c.foe_x, want.c.foe_y)
    ctx = dd.Context(W2, H2, fx, fy)
    for dev in (None, "cuda"):
        ev = dd.Events.of(w, device=dev)
        x, y, t = dd.dd_resample(ctx.h, ev, w.W, w.H, W2, H2, keep, seed)
        assert np.array_equal(x.cpu().numpy(), want.x) and np.array_equal(y.cpu().numpy(), want.y)
        assert np.array_equal(t.cpu().numpy(), want.t)
    ctx.close()
    return want


@pytest.mark.parametrize("W2,H2,keep,seed", [(160, 120, 0.25, 5), (640, 480, 1.0, 0), (320, 240, 0.5, 9),
                                             (97, 73, 0.1, 123)])
def test_resample_matches_oracle(W2, H2, keep, seed):
    check(window_config2(), W2, H2, keep, seed)


def test_resample_large_and_edge_windows():
    check(serve_config5(1, 120, n_scale=0.2), 160, 90, 0.25, 77)          # 1280x720 -> 160x90
    check(window_config1(), 346, 260, 1.0, 1)                              # identity
    check(make_window(5, 5, 2.0, 2.0, 400, 20, 100, 0.2, 0.5, 3), 2, 2, 1.0, 4)   # far-edge clamp
    check(make_window(64, 48, 32.0, 24.0, 0, 1, 0, 0.2, 0.5, 5), 16, 12, 0.25, 6)  # empty


def test_resample_rejects_events_outside_the_frame():
    w = window_config1()
    w.x[10] = w.W                                  # one event beyond the right edge
    ctx = dd.Context(80, 60, 40.0, 30.0)
    with pytest.raises(dd.DDError) as e:
        dd.dd_resample(ctx.h, dd.Events.of(w, device="cuda"), w.W, w.H, 80, 60)
    assert e.value.status == dd.DD_ERR_ARG
    with pytest.raises(dd.DDError):
        dd.dd_resample(ctx.h, dd.Events.of(window_config1(), device="cuda"), 346, 260, 80, 60, keep=1.5)
    ctx.close()


@pytest.mark.parametrize("pop_k", [1, 16])
def test_fast_solve_matches_oracle(pop_k):
    w = window_config2()
    want_win = O.resample(O.Window.of(w), 160, 120, 0.25, 5)
    want = O.solve(want_win, -1.0, 1.0, 1e-4, 0.0, pop_k, trace_cap=2048)
    fx, fy = dd.dd_resample_foe(w.W, w.H, w.foe_x, w.foe_y, 160, 120)
    ctx = dd.Context(160, 120, fx, fy, pop_k=pop_k)
    ev = ctx.resample(dd.Events.of(w, device="cuda"), w.W, w.H, keep=0.25, seed=5)
    got = ctx.solve(ev, -1.0, 1.0, 1e-4, 0.0, trace_cap=2048)
    for k in ("D_star", "K_hat", "gap_K", "nodes_expanded", "point_evals", "bound_evals", "cell_increments",
              "bound_increments", "rounds"):
        assert got[k] == want[k], k
    assert got["trace"] == want["trace"]
    assert abs(got["D_star"] - 0.35) <= 0.05
    ctx.close()


def test_time_span_of_a_batch():
    # Sec. 3.3 measures a batch's times from its earliest event: t0 = the
    # least timestamp, tau = greatest - least in binary32; the window so
    # described solves as the oracle's window [t0, t0 + tau].
    w = make_window(120, 90, 60.0, 45.0, 2000, 80, 500, 0.25, 0.4, 11, t0=3.25)
    ctx = dd.Context(w.W, w.H, w.foe_x, w.foe_y, pop_k=4)
    want = (float(w.t.min()), float(np.float32(w.t.max() - w.t.min())))
    for dev in (None, "cuda"):
        assert ctx.time_span(dd.Events.of(w, device=dev)) == want
    t0, tau = want
    got = ctx.solve(dd.Events.of(w, device="cuda").with_time(t0, tau))
    ref = O.solve(O.Window(w.W, w.H, w.foe_x, w.foe_y, w.x, w.y, w.t, t0, tau), -1.0, 1.0, 1e-4, 0.0, 4)
    for k in ("D_star", "K_hat", "gap_K", "nodes_expanded", "rounds"):
        assert got[k] == ref[k], k
    # several blocks of the device reduction; a non-finite timestamp is skipped
    g = torch.Generator(device="cuda").manual_seed(5)
    t = torch.rand(3_000_001, device="cuda", generator=g) * 7.0 + 1.0
    t[123] = float("nan")
    x = torch.zeros(t.shape[0], dtype=torch.int16, device="cuda")
    tn = t.cpu().numpy()
    fin = tn[np.isfinite(tn)]
    assert ctx.time_span(dd.Events(x, x, t, 0.0, 1.0)) == (float(fin.min()), float(np.float32(fin.max() - fin.min())))
    # no span, no events
    flat = torch.full((5,), 2.0, device="cuda")
    with pytest.raises(dd.DDError):
        ctx.time_span(dd.Events(x[:5], x[:5], flat, 0.0, 1.0))
    with pytest.raises(dd.DDError):
        ctx.time_span(dd.Events(x[:0], x[:0], flat[:0], 0.0, 1.0))
    ctx.close()
