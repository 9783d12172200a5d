"""Full-size parity: the largest windows of the batch, learned-warm-start,
serving and stream workloads, solved on the GPU in the configurations the
benchmarks run, against the oracle's Algorithm 1 on the same window.

These are the sizes where a bug of scale would show: 833k-event 1280x720
windows over D in [-1, 2] (long root segments, 1280-wide bands, split
merges, 64-bit counts), the 200k-event windows of the uneven batch, and the
trained model's warm starts on held-out windows.  Every key, count and the
expansion trace are compared exactly.
"""
import numpy as np
import pytest

import oracle as O
from synth import serve_config5
from synth.descent import batch_params3, batch_window3, stream_events5

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2209_13168_gb300 as dd  # noqa: E402

KEYS = ("D_star", "D_end", "K_hat", "gap_K", "nodes_expanded", "point_evals", "bound_evals", "event_warps",
        "cell_increments", "bound_increments", "rounds", "max_queue")
PARAMS5 = (-1.0, 2.0, 1e-4, 0.0)
TRACE = 1 << 14


def assert_same(got, want, what):
    for k in KEYS:
        assert got[k] == want[k], (what, k, got[k], want[k])


def serving_context():
    # the serving benchmark's context: the tuned 1280x720 batch knobs, pop 16
    from paper_2209_13168_gb300 import serve_bench
    return dd.Context.tuned(serve_bench.W, serve_bench.H, serve_bench.FX, serve_bench.FY, 100_000, mode="batch",
                            pop_k=16)


def test_heaviest_descent_window_alone_and_served_matches_oracle():
    # The last window of a descent (t = 18.8 s, D = 0.83, 833,333 events):
    # alone through dd_solve with its trace, then served beside three other
    # full-size windows of the other descents.
    heavy = serve_config5(0, 188)
    assert heavy.n == 833_333
    others = [serve_config5(1, 187), serve_config5(2, 150), serve_config5(3, 100)]
    ctx = serving_context()
    pop_k = ctx.cfg.pop_k
    ev = dd.Events.of(heavy, device="cuda")
    alone = ctx.solve(ev, *PARAMS5, trace_cap=TRACE)
    want = O.solve(O.Window.of(heavy), *PARAMS5, pop_k, trace_cap=TRACE)
    assert_same(alone, want, "alone")
    assert alone["trace_len"] == want["trace_len"] <= TRACE
    assert alone["trace"] == want["trace"]
    assert abs(alone["D_star"] - heavy.D_true) < 0.02

    solo = [ctx.solve(dd.Events.of(w, device="cuda"), *PARAMS5) for w in others]
    srv = dd.Server(ctx, max_slots=4, max_events=1 << 20)
    t0 = dd.Server.clock() + 0.005
    evs = [ev] + [dd.Events.of(w, device="cuda" if i % 2 else None) for i, w in enumerate(others)]
    tickets = [srv.submit(e, PARAMS5, t0 + 0.001 * i) for i, e in enumerate(evs)]
    got = [srv.wait(t) for t in tickets]
    st = srv.stats()
    srv.stop()
    assert st["peak_busy"] >= 2                   # the heavy window shared its rounds
    assert_same(got[0], want, "served")
    for r, s, w in zip(got[1:], solo, others):
        assert_same(r, s, "served vs alone")
    # one of the others against the oracle as well (200k events at t = 15 s)
    assert_same(got[2], O.solve(O.Window.of(others[1]), *PARAMS5, pop_k), "served 2")
    ctx.close()


def test_full_size_stream_windows_match_oracle():
    # Three 0.2 s windows of a full-size continuous descent stream from
    # t = 15 s (about 200k events each), in the stream benchmark's context.
    x, y, t = stream_events5(2, 150, 154)
    ev = dd.Events(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), torch.from_numpy(t).cuda(), 0.0, 1.0)
    ctx = dd.Context.tuned(1280, 720, 640.0, 360.0, x.shape[0] // 2, mode="batch", pop_k=16)
    n_win, tau, hop = 3, np.float32(0.2), 0.1
    rc, res, _, first = ctx.stream_solve(ev, 15.0, float(tau), hop, n_win, PARAMS5)
    assert rc == dd.DD_OK
    for k in range(n_win):
        t0 = np.float32(15.0 + hop * k)
        d = (t - t0).astype(np.float32)
        idx = np.nonzero((d >= 0) & (d <= tau))[0]
        f, n = int(idx[0]), idx.size
        assert first[k] == f and n > 150_000
        win = O.Window(1280, 720, 640.0, 360.0, x[f:f + n], y[f:f + n], t[f:f + n], float(t0), float(tau))
        want = O.solve(win, *PARAMS5, ctx.cfg.pop_k)
        for key in KEYS:
            if key not in ("event_warps", "max_queue"):
                assert res[k][key] == want[key], (k, key)
    ctx.close()


def test_largest_batch_windows_match_oracle():
    # The 256-window batch in the benchmark's configuration (tuned batch
    # knobs): its two largest windows (about 200k events), taken from the
    # batched result, against the oracle.
    params = batch_params3()
    ws = [batch_window3(i, params) for i in range(256)]
    ctx = dd.Context.tuned(640, 480, 320.0, 240.0, sum(w.n for w in ws) / len(ws), mode="batch")
    evs = [dd.Events.of(w, device="cuda") for w in ws]
    rc, res = ctx.solve_batch(evs)
    assert rc == dd.DD_OK
    order = np.argsort([w.n for w in ws])
    for i in (int(order[-1]), int(order[-2])):
        assert ws[i].n > 150_000
        want = O.solve(O.Window.of(ws[i]), -1.0, 1.0, 1e-4, 0.0, ctx.cfg.pop_k)
        assert_same(res[i], want, "batch window %d" % i)
    ctx.close()


def test_held_out_windows_with_the_trained_model_match_oracle():
    # Sixteen held-out windows (20k-100k events) solved as one batch from the
    # committed model's guesses, in the warm-start benchmark's context; the
    # oracle computes the same guess (features and network in binary32 with
    # the model's bfloat16 weights) and runs the warm-started Algorithm 1.
    from paper_2209_13168_gb300 import warm_start
    from synth import make_window
    from synth.descent import WARM_EVAL_SEED
    specs = warm_start.window_specs(16, WARM_EVAL_SEED)
    ws = [make_window(*s) for s in specs]
    ctx = warm_start.context()
    m = dd.Mlp(path=warm_start.DEFAULT_MODEL)
    ctx.set_warm_model(m)
    q = m.get_params()
    rc, res = ctx.solve_batch([dd.Events.of(w, device="cuda") for w in ws],
                              [warm_start.PARAMS + ("model",)] * len(ws))
    assert rc == dd.DD_OK
    for i, (w, r) in enumerate(zip(ws, res)):
        win = O.Window.of(w)
        f, _ = O.features(win)
        u, l = O.mlp_forward_f32(q, f)
        guess = O.warm_map(float(u), float(l), win.c.tau)
        want = O.solve(win, *warm_start.PARAMS, ctx.cfg.pop_k, warm=guess)
        assert_same(r, want, "held-out window %d" % i)
        assert (r["D_warm"], r["w_warm"]) == (np.float32(min(max(guess[0], -1.0), 1.0)), np.float32(guess[1]))
    ctx.close()
    m.close()
