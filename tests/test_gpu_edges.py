"""Edge cases of the frame and the window on the GPU against the oracle: the
FOE on the frame's corners, extreme aspect ratios, the largest frame, events
on the frame's edges and at both ends of the window, and the heaviest
full-size serving window (sampled hypotheses)."""
import numpy as np
import pytest

import oracle as O
from synth import make_window, serve_config5

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2209_13168_gb300 as dd  # noqa: E402

KEYS = ("D_star", "D_end", "K_hat", "gap_K", "nodes_expanded", "point_evals", "bound_evals", "cell_increments",
        "bound_increments", "rounds", "max_queue")


def check(w, Ds, lo, hi, want_iwe=True, solve_pop=4, **kw):
    win = O.Window.of(w)
    ctx = dd.Context(w.W, w.H, w.foe_x, w.foe_y, **kw)
    ev = dd.Events.of(w, device="cuda")
    K, S, N, img = ctx.contrast(ev, np.asarray(Ds, np.float32), want_iwe=want_iwe)
    for j, D in enumerate(np.asarray(Ds, np.float32)):
        k, s, n, im = O.contrast(win, float(D), want_iwe=want_iwe)
        assert (K[j], int(S[j]), int(N[j])) == (k, s, n), D
        if want_iwe:
            assert np.array_equal(img[j], im), D
    lo, hi = np.asarray(lo, np.float32), np.asarray(hi, np.float32)
    Kb, Sb, Nb, imb = ctx.bound(ev, lo, hi, want_iwe=want_iwe)
    for j in range(lo.size):
        k, s, n, im = O.bound(win, float(lo[j]), float(hi[j]), want_iwe=want_iwe)
        assert (Kb[j], int(Sb[j]), int(Nb[j])) == (k, s, n), (lo[j], hi[j])
        if want_iwe:
            assert np.array_equal(imb[j], im), (lo[j], hi[j])
    ctx.close()
    if solve_pop:
        ctx = dd.Context(w.W, w.H, w.foe_x, w.foe_y, pop_k=solve_pop, **kw)
        got = ctx.solve(ev, trace_cap=4096)
        want = O.solve(win, -1.0, 1.0, 1e-4, 0.0, solve_pop, trace_cap=4096)
        for k in KEYS:
            assert got[k] == want[k], k
        assert got["trace"] == want["trace"]
        ctx.close()


@pytest.mark.parametrize("foe", [(0.0, 0.0), (50.0, 40.0), (0.0, 40.0), (50.0, 0.0), (25.0, 0.0)])
def test_foe_on_the_frame_corners_and_edges(foe):
    w = make_window(50, 40, foe[0], foe[1], 1500, 60, 300, 0.3, 0.5, 21)
    check(w, [-1.0, 0.0, 0.3, 1.0], [-1.0, 0.25], [1.0, 0.35])


@pytest.mark.parametrize("W,H", [(4096, 24), (24, 4096)])
def test_extreme_aspect_ratios(W, H):
    w = make_window(W, H, W / 2.0, H / 2.0, 3000, 120, 500, 0.4, 0.4, 31)
    check(w, [-0.5, 0.4, 1.0], [-1.0, 0.39], [1.0, 0.41], want_iwe=True, band_rows=1 if H > W else 0)


def test_largest_frame():
    # 4096 x 4096 (the largest frame the boundary accepts): keys and images of
    # a few hypotheses and bounds; no full solve (each oracle step touches
    # 16.7M cells).
    w = make_window(4096, 4096, 2048.0, 2048.0, 16000, 400, 4000, 0.35, 0.3, 41)
    check(w, [0.0, 0.35], [0.3], [0.4], want_iwe=True, solve_pop=0, max_splits=1)
    check(w, [-1.0, 1.0], [-1.0, 0.349], [1.0, 0.351], want_iwe=False, solve_pop=0, max_splits=1)


def test_the_ends_of_the_search_domain():
    # D tau at both ends of the accepted domain, -64 and 3/4 (where the
    # bound's widening is still proven to hold): keys and images at the ends,
    # bounds reaching them, and a search whose interval ends at 3/4.
    w = make_window(64, 48, 32.0, 24.0, 1500, 60, 300, 0.5, 0.5, 61)
    assert np.float32(w.tau) == np.float32(0.5)
    check(w, [-128.0, -1.0, 1.5], [-128.0, 1.25, 1.4999], [-127.0, 1.5, 1.5], solve_pop=0)
    win = O.Window.of(w)
    ev = dd.Events.of(w, device="cuda")
    for pop in (1, 8):
        ctx = dd.Context(w.W, w.H, w.foe_x, w.foe_y, pop_k=pop)
        got = ctx.solve(ev, -2.0, 1.5, 1e-4, 0.0, trace_cap=4096)
        want = O.solve(win, -2.0, 1.5, 1e-4, 0.0, pop, trace_cap=4096)
        for k in KEYS:
            assert got[k] == want[k], (k, pop)
        assert got["trace"] == want["trace"]
        ctx.close()


def test_events_on_the_frame_edges_and_at_the_window_ends():
    w = make_window(64, 48, 31.5, 23.5, 2000, 80, 400, 0.3, 0.5, 51, t0=2.0)
    rng = np.random.default_rng(3)
    idx = rng.choice(w.n, 400, replace=False)
    cx = np.array([0, 63, 0, 63], np.int16)
    cy = np.array([0, 0, 47, 47], np.int16)
    w.x[idx[:100]] = cx[np.arange(100) % 4]             # the four corner pixels
    w.y[idx[:100]] = cy[np.arange(100) % 4]
    w.x[idx[100:200]] = 0                                # left and right columns
    w.x[idx[200:300]] = 63
    w.y[idx[300:400]] = 47                               # bottom row
    w.t[idx[:200]] = np.float32(2.0)                     # t = t0
    w.t[idx[200:400]] = np.float32(np.float32(2.0) + np.float32(0.5))   # t - t0 = tau in binary32
    assert np.all((w.t - np.float32(w.t0)).astype(np.float32) <= np.float32(w.tau))
    check(w, [-1.0, -0.3, 0.0, 0.3, 1.0], [-1.0, 0.2, 0.29], [1.0, 0.4, 0.31])


def test_heaviest_full_size_serving_window_sampled():
    # The last window of a 1280x720 descent at full size (833k events), in the
    # bench's serving configuration (pop 16): keys at sampled hypotheses and
    # bounds, against the oracle one by one.
    w = serve_config5(0, 188)
    assert w.n > 800_000
    win = O.Window.of(w)
    ctx = dd.Context(w.W, w.H, w.foe_x, w.foe_y, pop_k=16)
    ev = dd.Events.of(w, device="cuda")
    Ds = np.array([0.0, w.D_true, 1.9], np.float32)
    K, S, N, _ = ctx.contrast(ev, Ds)
    for j, D in enumerate(Ds):
        assert (K[j], int(S[j]), int(N[j])) == O.contrast(win, float(D))[:3]
    lo = np.array([-1.0, w.D_true - 0.01], np.float32)
    hi = np.array([2.0, w.D_true + 0.01], np.float32)
    Kb, Sb, Nb, _ = ctx.bound(ev, lo, hi)
    for j in range(2):
        assert (Kb[j], int(Sb[j]), int(Nb[j])) == O.bound(win, float(lo[j]), float(hi[j]))[:3]
    # the solve's certificate holds for the oracle's contrast at its answer
    r = ctx.solve(ev, -1.0, 2.0, 1e-4, 0.0)
    assert O.contrast(win, r["D_star"])[0] == r["K_hat"]
    assert abs(r["D_star"] - w.D_true) < 0.01
    ctx.close()
