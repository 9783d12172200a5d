"""Serving benchmark: concurrent descents through the continuous-batching
server (dd_serve_*).

Each of n_streams simulated descents at 1280x720 produces one 0.2 s window
every 0.1 s of flight (189 windows from t = 0 to 18.8 s; divergence rising
from 0.05 to 0.83 s^-1, 50k to 800k events, 15% noise).  Windows reach the
server as a Poisson process per stream at an offered rate (windows per
second per stream; 10 is real time), are admitted into free slots between
rounds, and are solved exactly over D in [-1, 2].  Reported: latency from
arrival to result (p50, p99, max), throughput, and whether each served
result equals the solve of the same window alone.

    python -m paper_2209_13168_gb300.serve_bench --rate 40 --streams 4
"""
import argparse
import json
import math
import time

import numpy as np

import paper_2209_13168_gb300 as dd

W, H, FX, FY = 1280, 720, 640.0, 360.0
PARAMS = (-1.0, 2.0, 1e-4, 0.0)
WINDOWS_PER_STREAM = 189


def make_windows(n_streams, per_stream=WINDOWS_PER_STREAM, n_scale=1.0):
    """Device-resident windows [(stream, w, GpuWindow)] of the descents."""
    from synth.descent import serve_spec5
    from synth.gpu import make_window_gpu
    return [(s, w, make_window_gpu(serve_spec5(s, w, n_scale))) for s in range(n_streams) for w in range(per_stream)]


def arrivals(n_streams, per_stream, rate_hz, seed=5):
    """Poisson arrival offsets (seconds) per (stream, window): exponential gaps
    of mean 1/rate, one process per stream."""
    rng = np.random.default_rng(seed)
    out = {}
    for s in range(n_streams):
        t = np.cumsum(rng.exponential(1.0 / rate_hz, per_stream))
        for w in range(per_stream):
            out[(s, w)] = float(t[w])
    return out


def to_host(win):
    """Pinned host copies of a device window's arrays (for the end-to-end run)."""
    return (win.x.cpu().pin_memory(), win.y.cpu().pin_memory(), win.t.cpu().pin_memory())


def run(rate_hz=40.0, n_streams=4, per_stream=WINDOWS_PER_STREAM, slots=16, pop_k=16, host=False, check=16,
        windows=None, ctx=None, warm=None, log=None):
    """Serve every window once at the offered rate; returns the measurements."""
    import torch
    own_ctx = ctx is None
    if own_ctx:
        ctx = dd.Context.tuned(W, H, FX, FY, 100_000, mode="batch", pop_k=pop_k)
    if windows is None:
        windows = make_windows(n_streams, per_stream)
    E = max(w.n for _, _, w in windows)
    params = PARAMS + (warm,)
    evs = {}
    for s, k, w in windows:
        if host:
            x, y, t = to_host(w)
            evs[(s, k)] = dd.Events(x, y, t, w.t0, w.tau)
        else:
            evs[(s, k)] = dd.Events.of(w)
    torch.cuda.synchronize()
    srv = dd.Server(ctx, max_slots=slots, max_events=E)
    arr = arrivals(n_streams, per_stream, rate_hz)
    order = sorted(arr, key=lambda key: arr[key])
    t0 = dd.Server.clock() + 0.05
    tickets = {key: srv.submit(evs[key], params, t0 + arr[key]) for key in order}
    res = {key: srv.wait(tickets[key]) for key in order}
    t_end = dd.Server.clock()
    st = srv.stats()
    srv.stop()
    lat = np.array([res[k]["latency_s"] for k in order])
    first = t0 + arr[order[0]]
    n_ev = sum(w.n for _, _, w in windows)
    out = {"offered_hz_per_stream": rate_hz, "streams": n_streams, "windows": len(order), "slots": srv.slots,
           "pop_k": ctx.cfg.pop_k, "host_inputs": bool(host),
           "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
           "max_ms": float(lat.max() * 1e3),
           "throughput_windows_per_s": len(order) / (t_end - first),
           "offered_windows_per_s": n_streams * rate_hz,
           "events_per_s": n_ev / (t_end - first), "rounds": st["rounds"], "peak_busy": st["peak_busy"]}
    if check:
        # Served results must equal the solve of the same window alone.
        keys = [order[i] for i in np.linspace(0, len(order) - 1, min(check, len(order))).astype(int)]
        same = 0
        for key in keys:
            one = ctx.solve(evs[key], *PARAMS, warm=warm) if warm else ctx.solve(evs[key], *PARAMS)
            same += all(one[f] == res[key][f] for f in ("D_star", "K_hat", "gap_K", "nodes_expanded",
                                                          "cell_increments", "rounds"))
        out["identical_to_solo"] = "%d/%d" % (same, len(keys))
    if own_ctx:
        ctx.close()
    if log:
        log(json.dumps(out))
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--rate", type=float, nargs="+", default=[10.0, 40.0, 160.0])
    ap.add_argument("--streams", type=int, default=4)
    ap.add_argument("--per-stream", type=int, default=WINDOWS_PER_STREAM)
    ap.add_argument("--slots", type=int, default=16)
    ap.add_argument("--pop-k", type=int, default=16)
    ap.add_argument("--host", action="store_true", help="inputs in pinned host memory (copied at admission)")
    a = ap.parse_args()
    import torch
    torch.cuda.set_device(0)
    ws = make_windows(a.streams, a.per_stream)
    ctx = dd.Context.tuned(W, H, FX, FY, 100_000, mode="batch", pop_k=a.pop_k)
    for r in a.rate:
        run(r, a.streams, a.per_stream, a.slots, host=a.host, windows=ws, ctx=ctx, log=print)
    ctx.close()


if __name__ == "__main__":
    main()
