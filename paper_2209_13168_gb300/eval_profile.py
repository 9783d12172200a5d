"""Per-round timing of the IWE evaluation kernel in one exact solve.

Runs the benchmark's single-window solve (the 640x480, 100,000-event window
with its tuned knobs; --window descent: the heaviest 1280x720 descent window,
833k events over D in [-1, 2]) with the library's launch timing on: the
rounds are launched from the host one per poll and each evaluation launch is
bracketed by CUDA events, so launch k of the solve is round k (0: the root).
Prints one JSON line: per-round device times and the solve's counts.

This is also the command the committed ncu captures of k_eval profile: with
`-k regex:k_eval -s <round> -c <n>` a capture selects rounds by number.

    python -m paper_2209_13168_gb300.eval_profile [--window config2|descent] [--warmup 1]
"""
import argparse
import json

import paper_2209_13168_gb300 as dd


def window(name):
    if name == "descent":
        from synth import serve_config5
        return serve_config5(0, 188), (-1.0, 2.0, 1e-4, 0.0), "batch", 16
    from synth import window_config2
    return window_config2(), (-1.0, 1.0, 1e-4, 0.0), "single", None


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--window", default="config2", choices=["config2", "descent"])
    ap.add_argument("--warmup", type=int, default=0, help="untimed graph solves first (not seen as rounds)")
    ap.add_argument("--fuse-span", type=int, default=None, help="dd_config.fuse_span (default: the tuned value)")
    for k in ("band-rows", "threads", "pop-k", "max-splits"):
        ap.add_argument("--" + k, type=int, default=None, help="override the tuned " + k.replace("-", "_"))
    a = ap.parse_args()
    import torch
    torch.cuda.set_device(0)
    w, params, mode, pop_k = window(a.window)
    kw = {"pop_k": pop_k} if pop_k else {}
    for k in ("fuse_span", "band_rows", "threads", "pop_k", "max_splits"):
        if getattr(a, k) is not None:
            kw[k] = getattr(a, k)
    ctx = dd.Context.tuned(w.W, w.H, w.foe_x, w.foe_y, w.n, mode=mode, **kw)
    ev = dd.Events.of(w, device="cuda")
    for _ in range(a.warmup):
        ctx.solve(ev, *params)
    ctx.set_timing(True)
    ctx.reset_stats()
    r = ctx.solve(ev, *params)
    ms = [float(x) for x in ctx.launch_times()]
    knobs = {k: getattr(ctx.cfg, k) for k in ("pop_k", "band_rows", "threads", "max_splits", "fuse_span")}
    ctx.close()
    out = {"window": a.window, "events": w.n, "knobs": knobs,
           "rounds": r["rounds"], "launches": len(ms), "eval_ms_total": sum(ms),
           "eval_ms_per_round": [round(x, 4) for x in ms],
           "point_evals": r["point_evals"], "bound_evals": r["bound_evals"],
           "cell_increments": r["cell_increments"], "bound_increments": r["bound_increments"],
           "nodes_expanded": r["nodes_expanded"], "D_star": r["D_star"]}
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
