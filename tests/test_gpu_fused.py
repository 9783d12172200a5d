"""Fused interval jobs: an expanded interval's centre and both halves
evaluated in one pass over a band's events (stable events counted once for
all three, the rest per task) must give exactly the keys, counts and traces
of three separate passes -- the oracle's.

The fusing threshold is a schedule knob (dd_config.fuse_span): never, the
default, wide, and every split interval (which also drives bands whose
unstable events overflow the list into the three-pass fallback).
"""
import pytest

import oracle as O
from synth import make_window, window_config1, window_config2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2209_13168_gb300 as dd  # noqa: E402

KEYS = ("D_star", "D_end", "K_hat", "gap_K", "nodes_expanded", "point_evals", "bound_evals", "event_warps",
        "cell_increments", "bound_increments", "rounds", "max_queue")
SPANS = (-1, 25, 200, 1_000_000)


def check(got, want):
    for k in KEYS:
        assert got[k] == want[k], (k, got[k], want[k])
    assert got["trace"] == want["trace"]


@pytest.mark.parametrize("fuse", SPANS)
def test_config2_solve_with_fused_intervals(fuse):
    w = window_config2()
    want = O.solve(O.Window.of(w), -1.0, 1.0, 1e-4, 0.0, 64, trace_cap=4096)
    ctx = dd.Context(w.W, w.H, w.foe_x, w.foe_y, pop_k=64, band_rows=20, max_splits=16, fuse_span=fuse)
    got = ctx.solve(dd.Events.of(w, device="cuda"), trace_cap=4096)
    check(got, want)
    ctx.close()


@pytest.mark.parametrize("fuse", SPANS)
@pytest.mark.parametrize("pop_k", [1, 8])
def test_config1_solve_with_fused_intervals(fuse, pop_k):
    w = window_config1()
    want = O.solve(O.Window.of(w), -1.0, 1.0, 1e-4, 0.0, pop_k, trace_cap=4096)
    ctx = dd.Context(w.W, w.H, w.foe_x, w.foe_y, pop_k=pop_k, fuse_span=fuse)
    got = ctx.solve(dd.Events.of(w, device="cuda"), trace_cap=4096)
    check(got, want)
    ctx.close()


@pytest.mark.parametrize("variant", [{"polarity": 1}, {"warp_to_start": 1}, {"polarity": 1, "warp_to_start": 1}])
def test_fused_intervals_with_objective_variants(variant):
    w = make_window(320, 240, 160.0, 120.0, 12000, 350, 4000, 0.3, 0.3, seed=4242)
    win = O.Window.of(w, t_ref=0.0 if variant.get("warp_to_start") else None,
                      polarity=bool(variant.get("polarity")))
    want = O.solve(win, -1.0, 1.0, 1e-4, 0.0, 16, trace_cap=4096)
    for fuse in (25, 1_000_000):
        ctx = dd.Context(w.W, w.H, w.foe_x, w.foe_y, pop_k=16, fuse_span=fuse, **variant)
        got = ctx.solve(dd.Events.of(w, device="cuda", polarity=bool(variant.get("polarity"))), trace_cap=4096)
        check(got, want)
        ctx.close()


def test_fused_intervals_in_a_batch():
    ws = [make_window(200, 150, 100.0, 75.0, 3000 + 2500 * i, 90 + 60 * i, 900, 0.1 + 0.12 * i, 0.25 + 0.05 * i,
                      seed=900 + i) for i in range(5)]
    for fuse in (25, 1_000_000):
        ctx = dd.Context(200, 150, 100.0, 75.0, pop_k=8, fuse_span=fuse)
        rc, res = ctx.solve_batch([dd.Events.of(w, device="cuda") for w in ws])
        assert rc == dd.DD_OK
        for w, r in zip(ws, res):
            want = O.solve(O.Window.of(w), -1.0, 1.0, 1e-4, 0.0, 8)
            for k in KEYS:
                assert r[k] == want[k], (fuse, k)
        ctx.close()
