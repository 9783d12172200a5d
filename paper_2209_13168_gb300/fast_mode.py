"""The paper's fast mode (resized and resampled windows) against full
resolution: time per exact solve and divergence error on synthetic descent
windows whose true D is known.

    python -m paper_2209_13168_gb300.fast_mode
"""
import json
import time

import numpy as np

import paper_2209_13168_gb300 as dd

def evaluate(windows, W2, H2, keep=0.25, seed=0, pop_k=None, reps=3, gamma=0.0, log=None):
    """Full-resolution vs fast-mode solves of `windows` (device-resident, one
    geometry): mean time per window (the fast mode includes its pre-pass)
    and mean |D* - D_true|.  gamma: Algorithm 1's stopping gap (contrast
    units; 0 = certified to the 1e-4 leaf width, the paper's runs used 0.025)."""
    PARAMS = (-1.0, 2.0, 1e-4, gamma)
    import torch
    w0 = windows[0]
    n_mean = sum(w.n for w in windows) // len(windows)
    kw = {"pop_k": pop_k} if pop_k else {}       # None: each frame's tuned knobs
    full = dd.Context.tuned(w0.W, w0.H, w0.foe_x, w0.foe_y, n_mean, mode="single", **kw)
    fx, fy = dd.dd_resample_foe(w0.W, w0.H, w0.foe_x, w0.foe_y, W2, H2)
    fast = dd.Context.tuned(W2, H2, fx, fy, int(n_mean * keep), mode="single", **kw)
    evs = [dd.Events.of(w) for w in windows]

    def run_full():
        return [full.solve(e, *PARAMS) for e in evs]

    def run_fast():
        return [fast.solve(fast.resample(e, w0.W, w0.H, keep, seed), *PARAMS) for e in evs]

    out = {}
    for name, fn in (("full", run_full), ("fast", run_fast)):
        res = fn()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            res = fn()
        dt = (time.perf_counter() - t0) / reps / len(evs)
        err = [abs(r["D_star"] - w.D_true) for r, w in zip(res, windows)]
        out[name] = {"ms_per_window": dt * 1e3, "mean_abs_err_D": float(np.mean(err)),
                     "max_abs_err_D": float(np.max(err)), "mean_nodes": float(np.mean([r["nodes_expanded"] for r in res]))}
    out["speedup"] = out["full"]["ms_per_window"] / out["fast"]["ms_per_window"]
    out["knobs"] = {name: {k: getattr(c.cfg, k) for k in ("pop_k", "band_rows", "threads", "max_splits", "fuse_span")}
                    for name, c in (("full", full), ("fast", fast))}
    out["frame"] = "%dx%d -> %dx%d, keep %.2f" % (w0.W, w0.H, W2, H2, keep)
    out["gamma"] = gamma
    out["windows"] = len(windows)
    full.close()
    fast.close()
    if log:
        log(json.dumps(out))
    return out


def descent_windows(stream=0, step=10):
    """Every `step`-th window of one 1280x720 serving descent, on the GPU."""
    from synth.descent import serve_spec5
    from synth.gpu import make_window_gpu
    return [make_window_gpu(serve_spec5(stream, k)) for k in range(0, 189, step)]


def main():
    import torch
    torch.cuda.set_device(0)
    ws = descent_windows()
    for gamma in (0.0, 0.025):
        evaluate(ws, 160, 90, gamma=gamma, log=print)


if __name__ == "__main__":
    main()
