"""Training and evaluation of the learned warm start.

Windows of 640x480 frames with 20k-100k events (descent windows with
uneven event counts, noise fractions and lengths) are generated on the GPU,
labelled by the exact batch solver (u* = D* tau), reduced to their
features, and the network is trained with the CUDA Adam step.  Evaluation
solves held-out windows twice, from the centre and from the model's guess,
and compares nodes, rounds, time and the certified optimum.

    python -m paper_2209_13168_gb300.warm_start train --windows 200000 --out model.bin
    python -m paper_2209_13168_gb300.warm_start eval --model model.bin --windows 4096
"""
import argparse
import json
import math
import os
import time

import numpy as np

import paper_2209_13168_gb300 as dd

DEFAULT_MODEL = os.path.join(os.path.dirname(os.path.abspath(__file__)), "warm_start_640x480.bin")
W, H, FX, FY = 640, 480, 320.0, 240.0
PARAMS = (-1.0, 1.0, 1e-4, 0.0)
CHUNK = 256


def window_specs(n_windows, seed):
    """make_window arguments of n_windows warm-start windows from seed base `seed`."""
    from synth.descent import batch_params4, batch_spec3
    p = batch_params4(n_windows, seed)
    return [batch_spec3(i, p, seed=seed) for i in range(n_windows)]


def gpu_windows(specs):
    from synth.gpu import make_window_gpu
    return [make_window_gpu(s) for s in specs]


def context(pop_k=16):
    return dd.Context.tuned(W, H, FX, FY, 50_000, mode="batch", pop_k=pop_k)


def label(ctx, specs, log=print):
    """(features [n][128], u* [n], D* [n], gap flags [n]) for the windows."""
    import torch
    feats, us, ds, gaps = [], [], [], []
    t0 = time.perf_counter()
    for c0 in range(0, len(specs), CHUNK):
        ws = gpu_windows(specs[c0:c0 + CHUNK])
        evs = [dd.Events.of(w) for w in ws]
        rc, res = ctx.solve_batch(evs, [PARAMS] * len(evs))
        if rc != dd.DD_OK:
            raise dd.DDError(rc, "labelling solve")
        feats.append(ctx.features(evs))
        tau = np.array([w.tau for w in ws], np.float64)
        D = np.array([r["D_star"] for r in res], np.float64)
        us.append(torch.from_numpy((D * tau).astype(np.float32)))
        ds.append(D)
        gaps.append(np.array([r["gap_K"] for r in res]) > 0)
        if log and (c0 // CHUNK) % 50 == 0:
            log("  labelled %d/%d windows (%.1f s)" % (c0 + len(ws), len(specs), time.perf_counter() - t0))
    return torch.cat(feats), torch.cat(us).cuda(), np.concatenate(ds), np.concatenate(gaps)


def train(n_windows=200_000, epochs=30, batch=256, lr=1e-3, seed=0, out=DEFAULT_MODEL, log=print):
    import torch
    from synth.descent import WARM_TRAIN_SEED
    torch.cuda.set_device(0)
    ctx = context()
    specs = window_specs(n_windows, WARM_TRAIN_SEED)
    t0 = time.perf_counter()
    X, U, _, _ = label(ctx, specs, log)
    t_label = time.perf_counter() - t0
    n_val = max(1, n_windows // 50)
    Xv, Uv = X[:n_val].contiguous(), U[:n_val].contiguous()
    Xt, Ut = X[n_val:].contiguous(), U[n_val:].contiguous()
    m = dd.Mlp(seed=seed)
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    loss = torch.empty(1, device="cuda")
    steps = epochs * (Xt.shape[0] // batch)
    step = 0
    t1 = time.perf_counter()
    hist = []
    for ep in range(epochs):
        perm = torch.randperm(Xt.shape[0], device="cuda", generator=g)
        for b0 in range(0, Xt.shape[0] - batch + 1, batch):
            idx = perm[b0:b0 + batch]
            rate = lr * 0.5 * (1.0 + math.cos(math.pi * step / max(1, steps)))   # cosine decay
            m.train_step(Xt[idx].contiguous(), Ut[idx].contiguous(), rate, loss)
            step += 1
        _, lv = m.grad(Xv, Uv)
        hist.append(float(lv.item()))
        if log:
            log("  epoch %d: validation loss %.4f" % (ep + 1, hist[-1]))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t1
    m.save(out)
    pred = m.forward(Xv).cpu().numpy()
    err = np.abs(pred[:, 0] - Uv.cpu().numpy())
    info = {"windows": n_windows, "epochs": epochs, "steps": step, "label_s": t_label, "train_s": t_train,
            "val_loss": hist[-1], "val_median_abs_err_Dtau": float(np.median(err)),
            "val_cover_frac": float(np.mean(err <= np.exp(pred[:, 1]))), "path": out}
    ctx.close()
    m.close()
    return info


def _solve_all(ctx, ws, warm):
    import torch
    evs = [dd.Events.of(w) for w in ws]
    params = [PARAMS + (wm,) for wm in warm] if isinstance(warm, list) else [PARAMS + (warm,)] * len(evs)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rc, res = ctx.solve_batch(evs, params)
    dt = time.perf_counter() - t0
    if rc != dd.DD_OK:
        raise dd.DDError(rc, "evaluation solve")
    return res, dt


def evaluate(model=DEFAULT_MODEL, n_windows=4096, pop_k=16, log=print):
    """Plain vs learned warm start on held-out windows, batch mode."""
    import torch
    from synth.descent import WARM_EVAL_SEED
    torch.cuda.set_device(0)
    ctx = context(pop_k)
    m = dd.Mlp(path=model)
    ctx.set_warm_model(m)
    specs = window_specs(n_windows, WARM_EVAL_SEED)
    tot = {"plain": [0, 0, 0.0], "learned": [0, 0, 0.0], "ideal": [0, 0, 0.0]}
    same_K = both_exact = consistent = 0
    err = []
    for c0 in range(0, n_windows, CHUNK):
        ws = gpu_windows(specs[c0:c0 + CHUNK])
        rp, tp = _solve_all(ctx, ws, None)
        rl, tl = _solve_all(ctx, ws, "model")
        # the best a guess can do: the certified answer itself, half-width 2^-10
        ri, ti = _solve_all(ctx, ws, [(r["D_star"], 2.0 ** -10) for r in rp])
        err += [abs(b["D_warm"] - a["D_star"]) * w.tau for a, b, w in zip(rp, rl, ws)]
        for a, b in zip(rp, rl):
            both = a["gap_K"] == 0 and b["gap_K"] == 0
            both_exact += both
            same_K += a["K_hat"] == b["K_hat"]
            consistent += (a["K_hat"] <= b["K_hat"] + b["gap_K"]) and (b["K_hat"] <= a["K_hat"] + a["gap_K"])
            if both and a["K_hat"] != b["K_hat"]:
                raise AssertionError("certified optima differ")
        for k, rr, t in (("plain", rp, tp), ("learned", rl, tl), ("ideal", ri, ti)):
            tot[k][0] += sum(r["nodes_expanded"] for r in rr)
            tot[k][1] += sum(r["rounds"] for r in rr)
            tot[k][2] += t
    ctx.close()
    m.close()
    out = {"windows": n_windows, "pop_k": pop_k,
           "nodes_plain": tot["plain"][0], "nodes_learned": tot["learned"][0],
           "rounds_plain": tot["plain"][1], "rounds_learned": tot["learned"][1],
           "solves_per_s_plain": n_windows / tot["plain"][2], "solves_per_s_learned": n_windows / tot["learned"][2],
           "nodes_ideal_guess": tot["ideal"][0], "rounds_ideal_guess": tot["ideal"][1],
           "solves_per_s_ideal_guess": n_windows / tot["ideal"][2],
           "median_abs_guess_err_Dtau": float(np.median(err)),
           "K_hat_identical": same_K, "both_certified_exact": both_exact, "certificates_consistent": consistent}
    if log:
        log(json.dumps(out))
    return out


def main():
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    t = sub.add_parser("train")
    t.add_argument("--windows", type=int, default=200_000)
    t.add_argument("--epochs", type=int, default=30)
    t.add_argument("--lr", type=float, default=1e-3)
    t.add_argument("--out", default=DEFAULT_MODEL)
    e = sub.add_parser("eval")
    e.add_argument("--model", default=DEFAULT_MODEL)
    e.add_argument("--windows", type=int, default=4096)
    e.add_argument("--pop-k", type=int, default=16)
    a = ap.parse_args()
    if a.cmd == "train":
        print(json.dumps(train(a.windows, a.epochs, lr=a.lr, out=a.out)))
    else:
        evaluate(a.model, a.windows, a.pop_k)


if __name__ == "__main__":
    main()
