"""The stream-wise estimation (Sec. 4.4) on a continuous synthetic descent:
windows of 0.2 s every 0.1 s over 19 s of a 1280x720 camera descending at
constant velocity (divergence 1/(20 - t)), solved in one batched launch per
stream, with the time to contact at each window's end (1/D_end) against the
truth (20 - t_end).  Divergence errors are reported as the paper's
comparison does (Sec. 6: absolute error in percent against the closest-in-time
truth, per window and after averaging the estimates over 0.5 s of time).

    python -m paper_2209_13168_gb300.stream
"""
import json
import time

import numpy as np

import paper_2209_13168_gb300 as dd

TAU, HOP = 0.2, 0.1
PARAMS = (-1.0, 2.0, 1e-4, 0.0)


def resolution_average(t_end, values, res=0.5):
    """Estimates averaged over bins of `res` seconds of their times: (mean
    time, mean value) per non-empty bin, in time order."""
    t_end = np.asarray(t_end, np.float64)
    values = np.asarray(values, np.float64)
    k = np.floor(t_end / res).astype(np.int64)
    out_t, out_v = [], []
    for b in np.unique(k):
        m = k == b
        out_t.append(float(t_end[m].mean()))
        out_v.append(float(values[m].mean()))
    return np.array(out_t), np.array(out_v)


def divergence_error_pct(D_est, t, t_contact=20.0):
    """Absolute error in percent of divergence estimates against the truth
    1/(t_contact - t) of the descent at their times."""
    D_true = 1.0 / (t_contact - np.asarray(t, np.float64))
    return 100.0 * np.abs(np.asarray(D_est, np.float64) - D_true) / D_true


def evaluate(stream=0, n_windows=188, pop_k=16, reps=2, n_scale=1.0, log=None):
    import torch
    from synth.gpu import make_stream_gpu
    x, y, t = make_stream_gpu(stream, 0, n_windows + 1, n_scale)
    ev = dd.Events(x, y, t, 0.0, 1.0)
    ctx = dd.Context.tuned(1280, 720, 640.0, 360.0, int(x.shape[0]) * 2 // max(1, n_windows), mode="batch",
                           pop_k=pop_k)
    rc, res, ttc, first = ctx.stream_solve(ev, 0.0, TAU, HOP, n_windows, PARAMS)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(reps):
        rc, res, ttc, first = ctx.stream_solve(ev, 0.0, TAU, HOP, n_windows, PARAMS)
    dt = (time.perf_counter() - t0) / reps
    t_end = np.array([float(np.float32(HOP * k)) + TAU for k in range(n_windows)])
    true_ttc = 20.0 - t_end
    rel = np.abs(ttc - true_ttc) / true_ttc
    D_end = np.array([r["D_end"] for r in res], np.float64)
    err = divergence_error_pct(D_end, t_end)
    tb, Db = resolution_average(t_end, D_end, 0.5)
    err_b = divergence_error_pct(Db, tb)
    n_ev = int(sum(r["event_warps"] // max(1, r["point_evals"] + r["bound_evals"]) for r in res))
    out = {"stream": stream, "windows": n_windows, "stream_events": int(x.shape[0]), "window_events": n_ev,
           "status": rc, "seconds": dt, "windows_per_s": n_windows / dt, "events_per_s": n_ev / dt,
           "ttc_rel_err_median": float(np.median(rel)), "ttc_rel_err_p90": float(np.percentile(rel, 90)),
           "ttc_rel_err_max": float(rel.max()),
           "div_err_pct_mean": float(err.mean()), "div_err_pct_median": float(np.median(err)),
           "div_err_pct_mean_0.5s": float(err_b.mean()), "bins_0.5s": int(tb.size)}
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
