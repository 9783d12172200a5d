"""Autotuner for the IWE tiling and the BnB schedule.

Times exact solves of sample windows on the current GPU for each candidate
(band rows, threads per block, intervals per round, split cap), then, with
the fastest of those, for each fusing threshold (how narrow an expanded
interval must be for its centre and both halves to run as one fused job:
the tasks evaluated per unit, one or three), and records the fastest in a
JSON table keyed by (frame geometry, event-count bucket, single-window or
batch, GPU name).  The knobs change only the schedule:
results are identical for every candidate (the table stores times, and the
tuner checks that every candidate returned the same keys).

    python -m paper_2209_13168_gb300.autotune --out tuned.json
"""
import argparse
import itertools
import json
import math
import os
import time

import paper_2209_13168_gb300 as dd

DEFAULT_TABLE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned_gb300.json")

CANDIDATES = {
    "band_rows": [8, 10, 12, 16, 18, 20, 24, 38],
    "threads": [128, 256, 512],
    "pop_k": [16, 32, 64],
    "max_splits": [4, 8, 16],
}
# second stage: dd_config.fuse_span (-1: never fuse, one task per unit)
FUSE_CANDIDATES = [-1, 10, 25, 40, 70]
KNOBS = ("band_rows", "threads", "pop_k", "max_splits", "fuse_span")


def size_bucket(n_events):
    """Event counts are bucketed by powers of two."""
    return int(2 ** max(0, round(math.log2(max(1, n_events)))))


def key(W, H, n_events, mode, gpu):
    return "%dx%d/n%d/%s/%s" % (W, H, size_bucket(n_events), mode, gpu)


def gpu_name():
    import torch
    return torch.cuda.get_device_name(0).replace(" ", "_")


def _time(fn, reps):
    import torch
    fn()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        out = fn()
    torch.cuda.synchronize()
    return (time.perf_counter() - t0) / reps, out


def tune(windows, mode="single", candidates=None, reps=3, log=print):
    """Best knobs for windows of one geometry (synth.Window objects)."""
    import torch
    cand = dict(CANDIDATES)
    if candidates:
        cand.update(candidates)
    w0 = windows[0]
    evs = [dd.Events.of(w, device="cuda") for w in windows]
    best, ref = None, None
    grid = list(itertools.product(cand["band_rows"], cand["threads"], cand["pop_k"],
                                  cand["max_splits"] if mode == "single" else [1], [0]))
    fuse = cand.get("fuse_span", FUSE_CANDIDATES)
    stage2 = False
    while grid:
        rows, thr, k, ms, fz = grid.pop(0)
        ctx = dd.Context(w0.W, w0.H, w0.foe_x, w0.foe_y, pop_k=k, band_rows=rows, threads=thr, max_splits=ms,
                         fuse_span=fz)
        if mode == "single":
            dt, out = _time(lambda: [ctx.solve(e) for e in evs], reps)
            keys = [r["K_hat"] for r in out]
            dt /= len(evs)
        else:
            dt, out = _time(lambda: ctx.solve_batch(evs), reps)
            keys = [r["K_hat"] for r in out[1]]
            dt /= len(evs)
        ctx.close()
        if ref is None:
            ref = keys
        assert keys == ref, "a schedule knob changed a result"
        log("  rows=%3d threads=%4d pop_k=%2d max_splits=%2d fuse_span=%d: %.3f ms per window"
            % (rows, thr, k, ms, fz, dt * 1e3))
        if best is None or dt < best["ms_per_window"] / 1e3:
            best = {"band_rows": rows, "threads": thr, "pop_k": k, "max_splits": ms, "fuse_span": fz,
                    "ms_per_window": dt * 1e3}
        if not grid and not stage2:              # then the fusing threshold, with the best of the rest
            stage2 = True
            grid = [(best["band_rows"], best["threads"], best["pop_k"], best["max_splits"], f) for f in fuse]
    torch.cuda.synchronize()
    return best


def load_table(path=DEFAULT_TABLE):
    try:
        return json.load(open(path))
    except (OSError, ValueError):
        return {}


def lookup(W, H, n_events, mode="single", path=DEFAULT_TABLE):
    """Tuned knobs for this geometry and size on this GPU (the nearest tuned
    event-count bucket of the same geometry and mode), or None."""
    try:
        name = gpu_name()
    except Exception:
        return None
    table = load_table(path)
    entry = table.get(key(W, H, n_events, mode, name))
    if not entry:
        prefix, suffix = "%dx%d/n" % (W, H), "/%s/%s" % (mode, name)
        near = [(abs(math.log2(int(k[len(prefix):-len(suffix)])) - math.log2(max(1, n_events))), k)
                for k in table if k.startswith(prefix) and k.endswith(suffix)]
        if not near:
            return None
        entry = table[min(near)[1]]
    return {k: entry[k] for k in KNOBS if k in entry}


class _Resampled:
    """A window given by device arrays (the fast mode's coarse window)."""

    def __init__(self, ev, W, H, foe_x, foe_y):
        self.x, self.y, self.t, self.t0, self.tau = ev.x, ev.y, ev.t, ev.c.t0, ev.c.tau
        self.W, self.H, self.foe_x, self.foe_y = W, H, foe_x, foe_y
        self.n = int(ev.c.n)


def fast_mode_windows(W2=160, H2=90, keep=0.25, step=20):
    """The fast mode's coarse windows of one 1280x720 descent (resampled on the GPU)."""
    from synth.descent import serve_spec5
    from synth.gpu import make_window_gpu
    fx, fy = dd.dd_resample_foe(1280, 720, 640.0, 360.0, W2, H2)
    rctx = dd.Context(W2, H2, fx, fy)
    out = []
    for k in range(0, 189, step):
        ev = rctx.resample(dd.Events.of(make_window_gpu(serve_spec5(0, k))), 1280, 720, keep=keep, seed=0)
        out.append(_Resampled(ev, W2, H2, fx, fy))
    rctx.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=DEFAULT_TABLE)
    ap.add_argument("--quick", action="store_true",
                    help="fewer candidates: the band heights, block sizes, pop widths and split caps that won on this GPU")
    ap.add_argument("--reps", type=int, default=3, help="timed repetitions per candidate (single windows)")
    ap.add_argument("--only", default=None, help="tune only the jobs whose name contains this (e.g. 1280x720)")
    args = ap.parse_args()
    import torch
    from synth import window_config1, window_config2
    from synth.descent import batch_params3, batch_window3
    torch.cuda.set_device(0)
    name = gpu_name()
    table = load_table(args.out)
    cand = None
    if args.quick:
        cand = {"band_rows": [12, 16, 20, 24], "threads": [256, 512], "pop_k": [16, 32, 64], "max_splits": [8, 16],
                "fuse_span": [-1, 15, 25, 40, 70]}
    from synth.descent import serve_config5
    jobs = [("single", [window_config1()]), ("single", [window_config2()])]
    params = batch_params3()
    jobs.append(("batch", [batch_window3(i, params) for i in range(256)]))
    # 1280x720 descent windows (serving, stream and fast-mode studies): five
    # windows of 100k-800k events one at a time, and a stream's 0.2 s windows
    jobs.append(("single", [serve_config5(0, k) for k in (20, 60, 100, 140, 180)]))
    jobs.append(("batch", [serve_config5(0, k, n_scale=0.5) for k in range(0, 189, 3)]))
    jobs.append(("single", fast_mode_windows()))
    for mode, ws in jobs:
        if args.only and args.only not in "%s %dx%d" % (mode, ws[0].W, ws[0].H):
            continue
        n = int(sum(w.n for w in ws) / len(ws))
        print("tuning %s %dx%d, %d windows of ~%d events" % (mode, ws[0].W, ws[0].H, len(ws), n), flush=True)
        best = tune(ws, mode, cand, reps=args.reps if mode == "single" else 3)
        best["windows"] = len(ws)
        best["events_per_window"] = n
        table[key(ws[0].W, ws[0].H, n, mode, name)] = best
        print("  best:", best, flush=True)
    with open(args.out + ".tmp", "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(args.out + ".tmp", args.out)


if __name__ == "__main__":
    main()
