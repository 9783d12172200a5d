"""The reference-time variant against the paper's warp.  Eq. 11 warps every
event to the window's end (t_ref = tau); warping to its start (t_ref = 0)
makes the scale 1 - D t linear in D, so the interval bound of Eqs. 14-19 is
the exact range of each event's scale rather than a range through a quotient.
Both solves are exact (certified to the leaf width); this compares the nodes
Algorithm 1 expands, its rounds, the time per window and the error against the
generator's D (the divergence at the window's start, the same parameter in
both warps).

    python -m paper_2209_13168_gb300.reference_time
"""
import json
import time

import numpy as np

import paper_2209_13168_gb300 as dd

VARIANTS = (("t_ref=tau", 0), ("t_ref=0", 1))


def compare(windows, params=(-1.0, 1.0, 1e-4, 0.0), pop_k=16, reps=3, batch=False):
    """Both warps on `windows` (device-resident, one geometry): per variant the
    time per window, mean nodes expanded and rounds, and |D* - D_true|."""
    import torch
    w0 = windows[0]
    evs = [dd.Events.of(w) for w in windows]
    out = {}
    for name, ref0 in VARIANTS:
        ctx = dd.Context(w0.W, w0.H, w0.foe_x, w0.foe_y, pop_k=pop_k, warp_to_start=ref0)
        if batch:
            def run():
                rc, res = ctx.solve_batch(evs, [params] * len(evs))
                if rc != dd.DD_OK:
                    raise dd.DDError(rc, "solve_batch")
                return res
        else:
            def run():
                return [ctx.solve(e, *params) for e in evs]
        res = run()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            res = run()
        dt = (time.perf_counter() - t0) / reps / len(evs)
        err = [abs(r["D_star"] - w.D_true) for r, w in zip(res, windows)]
        out[name] = {"ms_per_window": dt * 1e3,
                     "mean_nodes": float(np.mean([r["nodes_expanded"] for r in res])),
                     "mean_rounds": float(np.mean([r["rounds"] for r in res])),
                     "mean_bound_increments": float(np.mean([r["bound_increments"] for r in res])),
                     "mean_abs_err_D": float(np.mean(err)), "max_abs_err_D": float(np.max(err)),
                     "nodes": [r["nodes_expanded"] for r in res]}
        ctx.close()
    a, b = out["t_ref=tau"].pop("nodes"), out["t_ref=0"].pop("nodes")
    out["fewer_nodes_at_0"] = int(sum(y < x for x, y in zip(a, b)))
    out["more_nodes_at_0"] = int(sum(y > x for x, y in zip(a, b)))
    out["node_ratio"] = out["t_ref=0"]["mean_nodes"] / out["t_ref=tau"]["mean_nodes"]
    out["time_ratio"] = out["t_ref=0"]["ms_per_window"] / out["t_ref=tau"]["ms_per_window"]
    out["windows"] = len(windows)
    out["pop_k"] = pop_k
    out["mode"] = "batch" if batch else "one window per call"
    return out


def families():
    """Window families on the GPU: the 346x260 and 640x480 single-window
    workloads re-seeded, the uneven 256-window batch, and a 1280x720 descent."""
    from synth.descent import batch_params3, batch_spec3, serve_spec5
    from synth.gpu import make_window_gpu
    c1 = [make_window_gpu((346, 260, 173.0, 130.0, 3000, 150, 1000, 0.2, 0.5, 1000 + i)) for i in range(32)]
    c2 = [make_window_gpu((640, 480, 320.0, 240.0, 70000, 2000, 30000, 0.35, 0.3, 2000 + i)) for i in range(16)]
    p = batch_params3()
    c3 = [make_window_gpu(batch_spec3(i, p)) for i in range(256)]
    c5 = [make_window_gpu(serve_spec5(0, k)) for k in range(0, 189, 10)]
    return (("346x260, N 4000, D 0.2, tau 0.5; 32 seeds", c1, {}),
            ("640x480, N 100k, D 0.35, tau 0.3; 16 seeds", c2, {}),
            ("256 uneven 640x480 windows (N 5k-200k, D 0.05-0.8, tau 0.1-0.5), one batched solve", c3,
             {"batch": True}),
            ("every 10th window of a 1280x720 descent (D 0.05-0.83, tau 0.2, 50k-833k events)", c5,
             {"params": (-1.0, 2.0, 1e-4, 0.0)}))


def evaluate(reps=3, log=None):
    out = []
    for label, ws, kw in families():
        r = compare(ws, reps=reps, **kw)
        r["workload"] = label
        if log:
            log(json.dumps(r))
        out.append(r)
        del ws
    return out


def main():
    import torch
    torch.cuda.set_device(0)
    evaluate(log=print)


if __name__ == "__main__":
    main()
