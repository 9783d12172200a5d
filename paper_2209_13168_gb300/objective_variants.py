"""Objective variants against the paper's.  Eq. 11 warps every event to the
window's end (t_ref = tau) and Eq. 12 leaves polarity out.  Two variants:
warping to the window's start (t_ref = 0) makes the scale 1 - D t linear in
D, so the interval bound of Eqs. 14-19 is the exact range of each event's
scale rather than a range through a quotient; one image per polarity (the
contrasts of the two planes added) keeps events of opposite polarity from
sharing pixels.  Every solve is exact (certified to the leaf width); this
compares the nodes Algorithm 1 expands, its rounds, the time per window and
the error against the generator's D (the divergence at the window's start,
the same parameter under every variant).

    python -m paper_2209_13168_gb300.objective_variants
"""
import json
import time

import numpy as np

import paper_2209_13168_gb300 as dd

VARIANTS = (("paper", {}), ("t_ref=0", {"warp_to_start": 1}), ("polarity", {"polarity": 1}),
            ("polarity, t_ref=0", {"polarity": 1, "warp_to_start": 1}))


def compare(windows, params=(-1.0, 1.0, 1e-4, 0.0), pop_k=16, reps=3, batch=False, variants=VARIANTS):
    """Every variant on `windows` (device-resident with polarities, one
    geometry): per variant the time per window, mean nodes expanded and
    rounds, and |D* - D_true|; node and time ratios against the paper's."""
    import torch
    w0 = windows[0]
    out = {}
    nodes = {}
    for name, kw in variants:
        evs = [dd.Events.of(w, polarity=bool(kw.get("polarity"))) for w in windows]
        n_mean = sum(w.n for w in windows) // len(windows)
        ctx = dd.Context.tuned(w0.W, w0.H, w0.foe_x, w0.foe_y, n_mean, mode="batch" if batch else "single",
                               pop_k=pop_k, **kw)
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
        nodes[name] = [r["nodes_expanded"] for r in res]
        out[name] = {"ms_per_window": dt * 1e3,
                     "mean_nodes": float(np.mean(nodes[name])),
                     "mean_rounds": float(np.mean([r["rounds"] for r in res])),
                     "mean_bound_increments": float(np.mean([r["bound_increments"] for r in res])),
                     "mean_abs_err_D": float(np.mean(err)), "max_abs_err_D": float(np.max(err))}
        ctx.close()
    base = variants[0][0]
    for name, _ in variants[1:]:
        out[name]["node_ratio"] = out[name]["mean_nodes"] / out[base]["mean_nodes"]
        out[name]["time_ratio"] = out[name]["ms_per_window"] / out[base]["ms_per_window"]
        out[name]["fewer_nodes"] = int(sum(b < a for a, b in zip(nodes[base], nodes[name])))
        out[name]["more_nodes"] = int(sum(b > a for a, b in zip(nodes[base], nodes[name])))
    out["windows"] = len(windows)
    out["pop_k"] = pop_k
    out["mode"] = "batch" if batch else "one window per call"
    return out


def families():
    """Window families on the GPU, with polarities: the 346x260 and 640x480
    single-window workloads re-seeded, the uneven 256-window batch, and a
    1280x720 descent."""
    from synth.descent import batch_params3, batch_spec3, serve_spec5
    from synth.gpu import make_window_gpu

    def gen(spec):
        return make_window_gpu(spec, polarity=True)
    c1 = [gen((346, 260, 173.0, 130.0, 3000, 150, 1000, 0.2, 0.5, 1000 + i)) for i in range(32)]
    c2 = [gen((640, 480, 320.0, 240.0, 70000, 2000, 30000, 0.35, 0.3, 2000 + i)) for i in range(16)]
    p = batch_params3()
    c3 = [gen(batch_spec3(i, p)) for i in range(256)]
    c5 = [gen(serve_spec5(0, k)) for k in range(0, 189, 10)]
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
