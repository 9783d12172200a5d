"""Serving: continuous batching gives each window the result it gets alone.

Windows of several descents (the 1280x720 descent recipe at reduced event
counts) arrive at staggered times; the server admits them into free slots
between rounds, so they share evaluation launches with whatever else is in
flight.  Every result must be bit-identical to a single-window solve (same
pop width), and a sample to the oracle.
"""
import numpy as np
import pytest

import oracle as O
from synth import serve_config5

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2209_13168_gb300 as dd  # noqa: E402

KEYS = ("D_star", "D_end", "K_hat", "gap_K", "nodes_expanded", "point_evals", "bound_evals", "event_warps",
        "cell_increments", "bound_increments", "rounds", "max_queue")
PARAMS = (-1.0, 2.0, 1e-4, 0.0)


def windows(streams=3, per_stream=5, scale=0.02):
    return [serve_config5(s, 20 + 30 * w, n_scale=scale) for s in range(streams) for w in range(per_stream)]


def test_mixed_arrivals_match_solo_solves():
    ws = windows()
    ctx = dd.Context(1280, 720, 640.0, 360.0, pop_k=8)
    solo = [ctx.solve(dd.Events.of(w, device="cuda"), *PARAMS) for w in ws]
    srv = dd.Server(ctx, max_slots=4, max_events=1 << 16)
    t0 = dd.Server.clock() + 0.01
    evs = [dd.Events.of(w, device="cuda" if i % 2 else None) for i, w in enumerate(ws)]
    tickets = [srv.submit(e, PARAMS, t0 + 0.002 * i) for i, e in enumerate(evs)]
    got = [srv.wait(t) for t in tickets]
    st = srv.stats()
    srv.stop()
    for a, b in zip(got, solo):
        for k in KEYS:
            assert a[k] == b[k], k
        assert a["latency_s"] >= 0.0
    assert st["admitted"] == len(ws) and 1 <= st["peak_busy"] <= 4
    for i in (0, 7):
        want = O.solve(O.Window.of(ws[i]), *PARAMS, 8)
        assert got[i]["K_hat"] == want["K_hat"] and got[i]["nodes_expanded"] == want["nodes_expanded"]
    ctx.close()


def test_burst_waits_for_slots():
    ws = windows(streams=2, per_stream=4, scale=0.01)
    ctx = dd.Context(1280, 720, 640.0, 360.0, pop_k=4)
    srv = dd.Server(ctx, max_slots=2, max_events=1 << 15)
    tickets = [srv.submit(dd.Events.of(w, device="cuda"), PARAMS) for w in ws]
    got = [srv.wait(t) for t in tickets]
    st = srv.stats()
    srv.stop()
    assert st["peak_busy"] <= 2 and st["admitted"] == len(ws)
    for w, r in zip(ws, got):
        one = ctx.solve(dd.Events.of(w, device="cuda"), *PARAMS)
        for k in KEYS:
            assert r[k] == one[k], k
    ctx.close()


def test_capacity_and_malformed_windows():
    ws = windows(streams=1, per_stream=3, scale=0.01)
    ctx = dd.Context(1280, 720, 640.0, 360.0, pop_k=4)
    srv = dd.Server(ctx, max_slots=2, max_events=int(max(w.n for w in ws)))
    big = serve_config5(0, 150, n_scale=0.05)
    with pytest.raises(dd.DDError) as e:
        srv.submit(dd.Events.of(big, device="cuda"), PARAMS)
    assert e.value.status == dd.DD_ERR_CAPACITY
    ws[1].t[5] = np.float32(1.0)                 # outside its 0.2 s window
    tickets = [srv.submit(dd.Events.of(w, device="cuda"), PARAMS) for w in ws]
    r0 = srv.wait(tickets[0])
    with pytest.raises(dd.DDError) as e:
        srv.wait(tickets[1])
    assert e.value.status == dd.DD_ERR_ARG
    r2 = srv.wait(tickets[2])
    srv.stop()
    for w, r in ((ws[0], r0), (ws[2], r2)):
        assert r["K_hat"] == ctx.solve(dd.Events.of(w, device="cuda"), *PARAMS)["K_hat"]
    ctx.close()


def test_cancel_waiting_running_and_finished_requests():
    import time
    heavy = serve_config5(0, 188)                      # 833k events: hundreds of rounds at pop 1
    light = [serve_config5(1, 20 + 30 * i, n_scale=0.02) for i in range(3)]
    ctx = dd.Context(1280, 720, 640.0, 360.0, pop_k=1)
    solo = [ctx.solve(dd.Events.of(w, device="cuda"), *PARAMS) for w in light]
    srv = dd.Server(ctx, max_slots=2, max_events=1 << 20)
    # waiting: arrives in an hour, dropped
    far = srv.submit(dd.Events.of(light[0], device="cuda"), PARAMS, dd.Server.clock() + 3600.0)
    srv.cancel(far)
    with pytest.raises(dd.DDError) as e:
        srv.wait(far)
    assert e.value.status == dd.DD_ERR_CANCELLED
    # running: cancelled once admitted, stopped at the end of a round
    t_heavy = srv.submit(dd.Events.of(heavy, device="cuda"), PARAMS)
    t0 = time.perf_counter()
    while srv.stats()["admitted"] < 1 and time.perf_counter() - t0 < 10.0:
        time.sleep(1e-4)
    t_light = [srv.submit(dd.Events.of(w, device="cuda"), PARAMS) for w in light]
    srv.cancel(t_heavy)
    with pytest.raises(dd.DDError) as e:
        srv.wait(t_heavy)
    assert e.value.status == dd.DD_ERR_CANCELLED
    # the others, served beside it, are unaffected
    for t, want in zip(t_light, solo):
        got = srv.wait(t)
        for k in KEYS:
            assert got[k] == want[k], k
    # finished, not yet collected: nothing changes; unknown tickets are errors
    t_done = srv.submit(dd.Events.of(light[1], device="cuda"), PARAMS)
    time.sleep(0.5)
    srv.cancel(t_done)
    got = srv.wait(t_done)
    assert got["K_hat"] == solo[1]["K_hat"]
    with pytest.raises(dd.DDError):
        srv.cancel(t_done)                             # already collected
    srv.stop()
    ctx.close()


def test_host_inputs_are_uploaded_beside_running_windows():
    # Host-array windows are copied into their slots by the upload thread
    # while device-resident windows run; their searches start once the copy
    # has landed.  Every result equals the window solved alone; a host window
    # cancelled right after submission ends cancelled, whether it was still
    # waiting, uploading or running.
    heavy = serve_config5(0, 188)
    light = [serve_config5(1, 20 + 30 * i, n_scale=0.05) for i in range(4)]
    ctx = dd.Context(1280, 720, 640.0, 360.0, pop_k=8)
    solo = [ctx.solve(dd.Events.of(w, device="cuda"), *PARAMS) for w in light]
    srv = dd.Server(ctx, max_slots=3, max_events=1 << 20)
    tickets = [srv.submit(dd.Events.of(w, device=None if i % 2 == 0 else "cuda"), PARAMS)
               for i, w in enumerate(light)]
    t_heavy = srv.submit(dd.Events.of(heavy), PARAMS)
    srv.cancel(t_heavy)
    for t, want in zip(tickets, solo):
        got = srv.wait(t)
        for k in KEYS:
            assert got[k] == want[k], k
    with pytest.raises(dd.DDError) as e:
        srv.wait(t_heavy)
    assert e.value.status == dd.DD_ERR_CANCELLED
    # an uncancelled host window after it: served, identical to its solo solve
    want = ctx.solve(dd.Events.of(light[2], device="cuda"), *PARAMS)
    got = srv.wait(srv.submit(dd.Events.of(light[2]), PARAMS))
    for k in KEYS:
        assert got[k] == want[k], k
    srv.stop()
    ctx.close()
