"""Randomised parity: many small seeded configurations (frame sizes, FOE
anywhere in the frame including its edges, events on the FOE and on the
frame's edges, time origins, window lengths, search ranges across the
domain, every schedule knob, polarity planes, the start-of-window warp), each
compared with the oracle bit for bit: images at random hypotheses, bounds on
random intervals, and a traced search."""
import os

import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2209_13168_gb300 as dd  # noqa: E402

KEYS = ("D_star", "D_end", "K_hat", "gap_K", "nodes_expanded", "point_evals", "bound_evals", "cell_increments",
        "bound_increments", "rounds", "max_queue")


def case(seed):
    rng = np.random.default_rng(7_000 + seed)
    W, H = int(rng.integers(8, 200)), int(rng.integers(8, 150))
    fx = float(rng.choice([0.0, W, rng.uniform(0, W), np.floor(rng.uniform(0, W)) + 0.5]))
    fy = float(rng.choice([0.0, H, rng.uniform(0, H), float(rng.integers(0, H + 1))]))
    n = int(rng.integers(0, 3000))
    tau = float(np.float32(rng.uniform(0.05, 1.0)))
    t0 = float(np.float32(rng.uniform(-5.0, 5.0)))
    x = rng.integers(0, W, n).astype(np.int16)
    y = rng.integers(0, H, n).astype(np.int16)
    # some events on the FOE's pixel and on the frame's edges
    k = n // 10
    if k:
        x[:k] = min(W - 1, max(0, int(np.floor(fx + 0.5))))
        y[:k] = min(H - 1, max(0, int(np.floor(fy + 0.5))))
        x[k:2 * k] = rng.choice([0, W - 1], k)
        y[2 * k:3 * k] = rng.choice([0, H - 1], k)
    t = (np.float32(t0) + (rng.random(n) * tau).astype(np.float32)).astype(np.float32)
    t = np.minimum(t, np.float32(np.float32(t0) + np.float32(tau)))
    ok = (t - np.float32(t0)).astype(np.float32)
    t = np.where((ok >= 0) & (ok <= np.float32(tau)), t, np.float32(t0))
    p = rng.choice(np.array([-1, 1], np.int8), n)
    d_max = min(2.0, 0.74 / tau)
    D_lo = float(np.float32(rng.uniform(-2.0, 0.0)))
    D_hi = float(np.float32(rng.uniform(0.05, d_max)))
    knobs = dict(pop_k=int(rng.choice([1, 2, 7, 16, 64])), band_rows=int(rng.integers(1, H + 1)),
                 threads=int(rng.choice([32, 64, 96, 256, 512])), max_splits=int(rng.choice([1, 4, 16])),
                 host_loop=int(rng.integers(0, 2)), warp_to_start=int(rng.integers(0, 2)),
                 polarity=int(rng.integers(0, 2)))
    return dict(W=W, H=H, fx=fx, fy=fy, x=x, y=y, t=t, p=p, t0=t0, tau=tau, D_lo=D_lo, D_hi=D_hi, knobs=knobs,
                rng=rng)


# DD_FUZZ_SEEDS widens the sweep for a one-off run (1,000 extra seeds have
# been run that way, and 300 on the checked build, without a failure).
SEEDS = int(os.environ.get("DD_FUZZ_SEEDS", "120"))


@pytest.mark.parametrize("seed", range(SEEDS))
def test_random_configuration(seed):
    c = case(seed)
    kn = c["knobs"]
    win = O.Window(c["W"], c["H"], c["fx"], c["fy"], c["x"], c["y"], c["t"], c["t0"], c["tau"],
                   0.0 if kn["warp_to_start"] else None, c["p"] if kn["polarity"] else None)
    ctx = dd.Context(c["W"], c["H"], c["fx"], c["fy"], **kn)
    dev = "cuda" if seed % 2 else None
    if dev:
        ev = dd.Events(*(torch.from_numpy(a).cuda() for a in (c["x"], c["y"], c["t"])), c["t0"], c["tau"],
                       torch.from_numpy(c["p"]).cuda() if kn["polarity"] else None)
    else:
        ev = dd.Events(c["x"], c["y"], c["t"], c["t0"], c["tau"], c["p"] if kn["polarity"] else None)
    rng = c["rng"]
    Ds = np.float32(rng.uniform(c["D_lo"], c["D_hi"], 5))
    K, S, N, img = ctx.contrast(ev, Ds, want_iwe=True)
    for j, D in enumerate(Ds):
        k, s, n, im = O.contrast(win, float(D), want_iwe=True)
        assert (K[j], int(S[j]), int(N[j])) == (k, s, n), ("contrast", D)
        assert np.array_equal(img[j], im), ("image", D)
    a = np.float32(rng.uniform(c["D_lo"], c["D_hi"], 4))
    b = np.minimum(np.float32(a + np.float32(10.0) ** rng.uniform(-5, 0, 4)), np.float32(c["D_hi"]))
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    Kb, Sb, Nb, imb = ctx.bound(ev, lo, hi, want_iwe=True)
    for j in range(4):
        k, s, n, im = O.bound(win, float(lo[j]), float(hi[j]), want_iwe=True)
        assert (Kb[j], int(Sb[j]), int(Nb[j])) == (k, s, n), ("bound", lo[j], hi[j])
        assert np.array_equal(imb[j], im), ("bound image", lo[j], hi[j])
    got = ctx.solve(ev, c["D_lo"], c["D_hi"], 1e-4, 0.0, trace_cap=4096)
    want = O.solve(win, c["D_lo"], c["D_hi"], 1e-4, 0.0, kn["pop_k"], trace_cap=4096)
    for key in KEYS:
        assert got[key] == want[key], (key, got[key], want[key], kn)
    assert got["trace"] == want["trace"]
    ctx.close()
    assert dd.dd_check_flags()[0] == 0        # no index out of range (checked builds)
