"""Row splits in searches that share their rounds.

When several windows are searched together (a batch, or the serving loop's
busy slots), a round whose units leave the evaluation grid idle splits each
window's dense bound tasks by rows, every window taking its share of the
grid (no split merges: those buffers exist for a search alone).  A split is
a schedule choice: every key, count and node of every window must stay those
of the oracle's Algorithm 1 on that window alone, for any split cap.
"""
import pytest

import oracle as O
from synth import make_window, serve_config5, window_config2

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2209_13168_gb300 as dd  # noqa: E402

KEYS = ("D_star", "D_end", "K_hat", "gap_K", "nodes_expanded", "point_evals", "bound_evals", "event_warps",
        "cell_increments", "bound_increments", "rounds", "max_queue")


def assert_same(got, want, what):
    for k in KEYS:
        assert got[k] == want[k], (what, k, got[k], want[k])


@pytest.mark.parametrize("max_splits", [1, 4, 16])
def test_two_window_batch_with_row_splits_matches_oracle(max_splits):
    # A 100k-event window beside a small one: the first rounds leave most of
    # the grid idle, so the large window's bounds split by rows.
    big = window_config2()
    small = make_window(640, 480, 320.0, 240.0, 3000, 120, 900, 0.6, 0.2, seed=515)
    ctx = dd.Context(640, 480, 320.0, 240.0, pop_k=16, band_rows=20, max_splits=max_splits)
    rc, res = ctx.solve_batch([dd.Events.of(w, device="cuda") for w in (big, small)])
    assert rc == dd.DD_OK
    for w, r, name in ((big, res[0], "big"), (small, res[1], "small")):
        assert_same(r, O.solve(O.Window.of(w), -1.0, 1.0, 1e-4, 0.0, 16), name)
    ctx.close()


def test_served_windows_with_row_splits_match_oracle():
    # Two 1280x720 descent windows served together with splits allowed (and
    # fusing off, so that every interval's bounds are split candidates): each
    # result is the oracle's and the one the window gets alone.
    ws = [serve_config5(1, 120), serve_config5(2, 60)]
    ctx = dd.Context(1280, 720, 640.0, 360.0, pop_k=16, band_rows=16, max_splits=16, fuse_span=-1)
    params = (-1.0, 2.0, 1e-4, 0.0)
    srv = dd.Server(ctx, max_slots=2, max_events=1 << 19)
    t0 = dd.Server.clock() + 0.005
    tickets = [srv.submit(dd.Events.of(w, device="cuda" if i == 0 else None), params, t0) for i, w in enumerate(ws)]
    got = [srv.wait(t) for t in tickets]
    srv.stop()
    for w, r in zip(ws, got):
        assert_same(r, O.solve(O.Window.of(w), *params, 16), "served")
        assert_same(r, ctx.solve(dd.Events.of(w, device="cuda"), *params), "alone")
    ctx.close()


def test_batch_of_uneven_windows_with_row_splits():
    # Twelve windows of 500 to 40,000 events, 346x260: windows retire at
    # different rounds, so the share of the grid each remaining one takes
    # grows as the batch thins out.
    ws = [make_window(346, 260, 173.0, 130.0, 400 + 3300 * i, 20 + 30 * i, 100 + 600 * i, 0.1 + 0.06 * i,
                      0.15 + 0.03 * i, seed=2000 + i) for i in range(12)]
    ctx = dd.Context(346, 260, 173.0, 130.0, pop_k=8, max_splits=16)
    rc, res = ctx.solve_batch([dd.Events.of(w, device="cuda") for w in ws])
    assert rc == dd.DD_OK
    for i, (w, r) in enumerate(zip(ws, res)):
        assert_same(r, O.solve(O.Window.of(w), -1.0, 1.0, 1e-4, 0.0, 8), "window %d" % i)
    ctx.close()
