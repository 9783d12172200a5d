"""The stream-wise estimation (Sec. 4.4) on a continuous synthetic descent:
windows of 0.2 s every 0.1 s over 19 s of a 1280x720 camera descending at
constant velocity (divergence 1/(20 - t)), solved in one batched launch per
stream, with the time to contact at each window's end (1/D_end) against the
truth (20 - t_end).

    python -m paper_2209_13168_gb300.stream
"""
import json
import time

import numpy as np

import paper_2209_13168_gb300 as dd

TAU, HOP = 0.2, 0.1
PARAMS = (-1.0, 2.0, 1e-4, 0.0)


def evaluate(stream=0, n_windows=188, pop_k=16, reps=2, n_scale=1.0, log=None):
    import torch
    from synth.gpu import make_stream_gpu
    x, y, t = make_stream_gpu(stream, 0, n_windows + 1, n_scale)
    ev = dd.Events(x, y, t, 0.0, 1.0)
    ctx = dd.Context(1280, 720, 640.0, 360.0, pop_k=pop_k)
    rc, res, ttc, first = ctx.stream_solve(ev, 0.0, TAU, HOP, n_windows, PARAMS)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        rc, res, ttc, first = ctx.stream_solve(ev, 0.0, TAU, HOP, n_windows, PARAMS)
    dt = (time.perf_counter() - t0) / reps
    t_end = np.array([float(np.float32(HOP * k)) + TAU for k in range(n_windows)])
    true_ttc = 20.0 - t_end
    rel = np.abs(ttc - true_ttc) / true_ttc
    n_ev = int(sum(r["event_warps"] // max(1, r["point_evals"] + r["bound_evals"]) for r in res))
    out = {"stream": stream, "windows": n_windows, "stream_events": int(x.shape[0]), "window_events": n_ev,
           "status": rc, "seconds": dt, "windows_per_s": n_windows / dt, "events_per_s": n_ev / dt,
           "ttc_rel_err_median": float(np.median(rel)), "ttc_rel_err_p90": float(np.percentile(rel, 90)),
           "ttc_rel_err_max": float(rel.max())}
    ctx.close()
    if log:
        log(json.dumps(out))
    return out


def main():
    import torch
    torch.cuda.set_device(0)
    for s in range(4):
        evaluate(s, log=print)


if __name__ == "__main__":
    main()
