"""The per-polarity objective on the GPU against the oracle: one image per
polarity, contrasts added.  Images, keys, bounds and searches bit for bit,
through every entry point that takes events (single window, batch, stream,
serving), and with the start-of-window warp."""
import numpy as np
import pytest

import oracle as O
from synth import make_window, window_config1, window_config2, serve_config5
from synth.descent import batch_params3, batch_window3, stream_events5

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2209_13168_gb300 as dd  # noqa: E402

KEYS = ("D_star", "D_end", "K_hat", "gap_K", "nodes_expanded", "point_evals", "bound_evals", "cell_increments",
        "bound_increments", "rounds", "max_queue")


def ctx_for(w, **kw):
    return dd.Context(w.W, w.H, w.foe_x, w.foe_y, polarity=1, **kw)


@pytest.mark.parametrize("make", [window_config1, window_config2])
def test_images_with_polarity(make):
    w = make()
    win = O.Window.of(w, polarity=True)
    ctx = ctx_for(w)
    Ds = np.array([-1.0, -0.2, 0.0, 0.2, 0.35, 1.0], np.float32)
    for dev in (None, "cuda"):
        K, S, N, img = ctx.contrast(dd.Events.of(w, device=dev, polarity=True), Ds, want_iwe=True)
        for j, D in enumerate(Ds):
            k, s, n, im = O.contrast(win, float(D), want_iwe=True)
            assert (K[j], int(S[j]), int(N[j])) == (k, s, n), (D, dev)
            assert np.array_equal(img[j], im), (D, dev)
    lo = np.array([-1.0, 0.1, 0.3, 0.34], np.float32)
    hi = np.array([1.0, 0.2, 0.3001, 0.36], np.float32)
    Kb, Sb, Nb, imb = ctx.bound(dd.Events.of(w, device="cuda", polarity=True), lo, hi, want_iwe=True)
    for j in range(lo.size):
        k, s, n, im = O.bound(win, float(lo[j]), float(hi[j]), want_iwe=True)
        assert (Kb[j], int(Sb[j]), int(Nb[j])) == (k, s, n)
        assert np.array_equal(imb[j], im)
    ctx.close()


def test_one_polarity_equals_the_paper_objective():
    w = window_config2()
    w.p[:] = 1
    a = dd.Context(w.W, w.H, w.foe_x, w.foe_y, pop_k=16)
    b = ctx_for(w, pop_k=16)
    ra = a.solve(dd.Events.of(w, device="cuda"), trace_cap=2048)
    rb = b.solve(dd.Events.of(w, device="cuda", polarity=True), trace_cap=2048)
    for k in KEYS:
        assert ra[k] == rb[k], k
    assert ra["trace"] == rb["trace"]
    a.close()
    b.close()


@pytest.mark.parametrize("pop_k,warp_to_start", [(1, 0), (16, 0), (16, 1)])
def test_solve_with_polarity(pop_k, warp_to_start):
    for w in (window_config1(), window_config2()):
        ctx = ctx_for(w, pop_k=pop_k, warp_to_start=warp_to_start)
        got = ctx.solve(dd.Events.of(w, device="cuda", polarity=True), trace_cap=4096)
        win = O.Window.of(w, t_ref=0.0 if warp_to_start else None, polarity=True)
        want = O.solve(win, -1.0, 1.0, 1e-4, 0.0, pop_k, trace_cap=4096)
        for k in KEYS:
            assert got[k] == want[k], (k, got[k], want[k])
        assert got["trace"] == want["trace"]
        ctx.close()


def test_batch_with_polarity():
    params = batch_params3()
    ws = [batch_window3(i, params) for i in (142, 68, 62, 228)]       # the smallest windows
    ctx = dd.Context(640, 480, 320.0, 240.0, pop_k=8, polarity=1)
    rc, res = ctx.solve_batch([dd.Events.of(w, device="cuda", polarity=True) for w in ws])
    assert rc == dd.DD_OK
    for w, r in zip(ws, res):
        want = O.solve(O.Window.of(w, polarity=True), -1.0, 1.0, 1e-4, 0.0, 8)
        for k in KEYS:
            assert r[k] == want[k], k
    ctx.close()


@pytest.mark.parametrize("device", [None, "cuda"])
def test_stream_with_polarity(device):
    x, y, t, p = stream_events5(0, 100, 106, n_scale=0.02, with_polarity=True)
    if device is None:
        ev = dd.Events(x, y, t, 0.0, 1.0, p)
    else:
        ev = dd.Events(*(torch.from_numpy(a).cuda() for a in (x, y, t)), 0.0, 1.0, torch.from_numpy(p).cuda())
    ctx = dd.Context(1280, 720, 640.0, 360.0, pop_k=8, polarity=1)
    params = (-1.0, 2.0, 1e-4, 0.0)
    rc, res, ttc, first = ctx.stream_solve(ev, 10.0, 0.2, 0.1, 4, params)
    assert rc == dd.DD_OK
    for k in range(4):
        t0 = np.float32(10.0 + 0.1 * k)
        d = (t - t0).astype(np.float32)
        idx = np.nonzero((d >= 0) & (d <= np.float32(0.2)))[0]
        f, n = int(idx[0]), idx.size
        assert first[k] == f
        win = O.Window(1280, 720, 640.0, 360.0, x[f:f + n], y[f:f + n], t[f:f + n], float(t0), 0.2, None,
                       p[f:f + n])
        want = O.solve(win, *params, 8)
        for key in KEYS[:-1]:
            assert res[k][key] == want[key], (k, key)
    ctx.close()


def test_serving_with_polarity():
    ws = [serve_config5(s, 40, n_scale=0.02) for s in range(3)]
    params = (-1.0, 2.0, 1e-4, 0.0)
    ctx = dd.Context(1280, 720, 640.0, 360.0, pop_k=8, polarity=1)
    srv = dd.Server(ctx, max_slots=2, max_events=1 << 16)
    tickets = [srv.submit(dd.Events.of(w, device="cuda" if i % 2 else None, polarity=True), params)
               for i, w in enumerate(ws)]
    got = [srv.wait(tk) for tk in tickets]
    with pytest.raises(dd.DDError):                  # a polarity server needs the polarities
        srv.submit(dd.Events.of(ws[0], device="cuda"), params)
    srv.stop()
    for w, r in zip(ws, got):
        want = O.solve(O.Window.of(w, polarity=True), *params, 8)
        for k in KEYS[:-1]:
            assert r[k] == want[k], k
    ctx.close()


def test_polarity_arguments():
    w = make_window(64, 48, 32.0, 24.0, 400, 20, 100, 0.2, 0.5, 3)
    ctx = ctx_for(w)
    with pytest.raises(dd.DDError) as e:             # events without polarities
        ctx.solve(dd.Events.of(w, device="cuda"))
    assert e.value.status == dd.DD_ERR_ARG
    with pytest.raises(dd.DDError):
        ctx.contrast(dd.Events.of(w), np.array([0.1], np.float32))
    ctx.close()
    with pytest.raises(dd.DDError):                  # 2 x 4096 rows exceed the event sort's bins
        dd.Context(64, 4096, 32.0, 2048.0, polarity=1)
    with pytest.raises(dd.DDError):
        dd.Context(64, 48, 32.0, 24.0, polarity=2)
    # empty windows need no polarities
    e0 = make_window(64, 48, 32.0, 24.0, 0, 1, 0, 0.2, 0.5, 5)
    ctx = ctx_for(e0)
    K, S, N, _ = ctx.contrast(dd.Events.of(e0, device="cuda"), np.array([0.1], np.float32))
    assert K == [0] and int(N[0]) == 0
    ctx.close()
