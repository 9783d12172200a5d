"""Randomised parity of the batched solver: each case is one context with
random knobs (pop width, band rows, threads, split cap, host or graph loop,
polarity planes, the start-of-window warp) and a batch of windows that
differ in everything a window can differ in (event count, empty windows
included, time origin, length, search interval, tolerance, stopping gap and
a given warm start), host and device inputs mixed.  Every window's result
must equal the oracle's Algorithm 1 on that window alone, bit for bit."""
import os

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2209_13168_gb300 as dd  # noqa: E402

KEYS = ("D_star", "D_end", "K_hat", "gap_K", "nodes_expanded", "point_evals", "bound_evals", "event_warps",
        "cell_increments", "bound_increments", "rounds", "max_queue")


def window(rng, W, H, fx, fy, n):
    tau = float(np.float32(rng.uniform(0.05, 0.8)))
    t0 = float(np.float32(rng.uniform(-3.0, 3.0)))
    x = rng.integers(0, W, n).astype(np.int16)
    y = rng.integers(0, H, n).astype(np.int16)
    t = (np.float32(t0) + (rng.random(n) * tau).astype(np.float32)).astype(np.float32)
    ok = (t - np.float32(t0)).astype(np.float32)
    t = np.where((ok >= 0) & (ok <= np.float32(tau)), t, np.float32(t0)).astype(np.float32)
    p = rng.choice(np.array([-1, 1], np.int8), n)
    D_lo = float(np.float32(rng.uniform(-1.5, 0.0)))
    D_hi = float(np.float32(rng.uniform(0.05, min(1.5, 0.74 / tau))))
    tol = float(rng.choice([3e-5, 1e-4, 1e-3]))
    gamma = float(rng.choice([0.0, 0.0, 1e-3]))
    warm = None
    if rng.random() < 0.3:
        warm = (float(np.float32(rng.uniform(D_lo - 0.2, D_hi + 0.2))), float(np.float32(2.0 ** rng.integers(-12, 0))))
    return dict(x=x, y=y, t=t, p=p, t0=t0, tau=tau, params=(D_lo, D_hi, tol, gamma), warm=warm)


# DD_FUZZ_BATCHES widens the sweep for a one-off run (200 extra batches have
# been run that way, and 60 on the checked build, without a failure).
BATCHES = int(os.environ.get("DD_FUZZ_BATCHES", "30"))


@pytest.mark.parametrize("seed", range(BATCHES))
def test_random_batch(seed):
    rng = np.random.default_rng(9_100 + seed)
    W, H = int(rng.integers(16, 180)), int(rng.integers(16, 140))
    fx = float(rng.choice([W / 2.0, float(rng.integers(0, W + 1)), np.floor(rng.uniform(0, W)) + 0.5]))
    fy = float(rng.choice([H / 2.0, float(rng.integers(0, H + 1))]))
    knobs = dict(pop_k=int(rng.choice([1, 3, 8, 32])), band_rows=int(rng.integers(1, H + 1)),
                 threads=int(rng.choice([64, 128, 256, 512])), max_splits=int(rng.choice([1, 4, 16])),
                 host_loop=int(rng.integers(0, 2)), warp_to_start=int(rng.integers(0, 2)),
                 polarity=int(rng.integers(0, 2)))
    nw = int(rng.integers(2, 11))
    counts = [int(rng.integers(0, 2500)) for _ in range(nw)]
    if seed % 3 == 0:
        counts[int(rng.integers(0, nw))] = 0                     # an empty window in the batch
    ws = [window(rng, W, H, fx, fy, n) for n in counts]
    pol = bool(knobs["polarity"])
    evs = []
    for i, w in enumerate(ws):
        if i % 2:
            evs.append(dd.Events(*(torch.from_numpy(w[k]).cuda() for k in ("x", "y", "t")), w["t0"], w["tau"],
                                 torch.from_numpy(w["p"]).cuda() if pol else None))
        else:
            evs.append(dd.Events(w["x"], w["y"], w["t"], w["t0"], w["tau"], w["p"] if pol else None))
    params = [w["params"] + ((w["warm"],) if w["warm"] is not None else ()) for w in ws]
    ctx = dd.Context(W, H, fx, fy, **knobs)
    rc, res = ctx.solve_batch(evs, params)
    assert rc == dd.DD_OK, (rc, [r["status"] for r in res])
    for w, r in zip(ws, res):
        win = O.Window(W, H, fx, fy, w["x"], w["y"], w["t"], w["t0"], w["tau"],
                       0.0 if knobs["warp_to_start"] else None, w["p"] if pol else None)
        want = O.solve(win, *w["params"], knobs["pop_k"], warm=w["warm"])
        assert r["status"] == dd.DD_OK
        for k in KEYS:
            assert r[k] == want[k], (k, r[k], want[k], knobs, w["params"], w["warm"], int(w["x"].size))
    ctx.close()
    assert dd.dd_check_flags()[0] == 0        # no index out of range (checked builds)
