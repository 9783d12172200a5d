"""Learned warm start on the GPU against the oracle.

Features and the binary32 network are compared bit for bit (same binning,
same summation order), the backprop gradient within 1e-2 of the oracle's
binary64 gradient on the same bfloat16 weights, and every warm-started
search -- from a given guess or from the model -- bit for bit with the
oracle's warm-started Algorithm 1 (incumbent, keys, counts, traces).
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from synth import make_window, window_config1, window_config2, serve_config5

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2209_13168_gb300 as dd  # noqa: E402

KEYS = ("D_star", "D_end", "K_hat", "gap_K", "nodes_expanded", "point_evals", "bound_evals", "event_warps",
        "cell_increments", "bound_increments", "rounds", "max_queue")


def bf16_round(a):
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def random_params(seed, out_scale=1.0):
    rng = np.random.default_rng(seed)
    o = O.OFFSETS
    p = np.zeros(O.N_PARAMS, np.float32)
    p[o["W1"]:o["b1"]] = rng.normal(0, math.sqrt(2 / 128), 16384)
    p[o["b1"]:o["W2"]] = rng.normal(0, 0.05, 128)
    p[o["W2"]:o["b2"]] = rng.normal(0, math.sqrt(2 / 128), 16384)
    p[o["b2"]:o["W3"]] = rng.normal(0, 0.05, 128)
    p[o["W3"]:o["b3"]] = rng.normal(0, out_scale * math.sqrt(1 / 128), 256)
    p[o["b3"]:] = [0.08, -3.0]
    return p


def evaluated(p):
    """The parameters as the network evaluates them (weights in bfloat16)."""
    q = p.copy()
    o = O.OFFSETS
    for a, b in (("W1", "b1"), ("W2", "b2"), ("W3", "b3")):
        q[o[a]:o[b]] = bf16_round(q[o[a]:o[b]])
    return q


def small_windows():
    ws = [make_window(97, 61, 48.0, 30.0, 900, 45, 300, 0.3, 0.35, 9),
          make_window(97, 61, 48.0, 30.0, 20000, 500, 3000, -0.4, 0.25, 10),      # several chunks, ragged tail
          make_window(97, 61, 48.0, 30.0, 0, 1, 0, 0.3, 0.35, 11),                # empty
          make_window(97, 61, 48.0, 30.0, 40, 2, 7, 0.6, 0.5, 12, t0=3.25)]       # t0 offset
    return ws


# ---------------------------------------------------------------- features

def test_features_match_oracle():
    ws = small_windows()
    ctx = dd.Context(97, 61, 48.0, 30.0)
    evs = [dd.Events.of(w, device="cuda" if i % 2 else None) for i, w in enumerate(ws)]
    got = ctx.features(evs).cpu().numpy()
    for i, w in enumerate(ws):
        want, _ = O.features(O.Window.of(w))
        assert np.array_equal(got[i], want), i
    ctx.close()


@pytest.mark.parametrize("make", [window_config1, window_config2])
def test_features_match_oracle_config(make):
    w = make()
    ctx = dd.Context(w.W, w.H, w.foe_x, w.foe_y)
    got = ctx.features([dd.Events.of(w, device="cuda")]).cpu().numpy()[0]
    want, _ = O.features(O.Window.of(w))
    assert np.array_equal(got, want)
    ctx.close()


# ----------------------------------------------------------------- network

def test_params_roundtrip_and_bf16():
    m = dd.Mlp(seed=3)
    p = random_params(1)
    m.set_params(p)
    assert np.array_equal(m.get_params(), evaluated(p))
    m.close()


def test_forward_bit_exact_with_oracle():
    m = dd.Mlp()
    rng = np.random.default_rng(4)
    for s in range(3):
        p = random_params(10 + s, out_scale=4.0)
        m.set_params(p)
        q = evaluated(p)
        X = (rng.random((37, 128)) * 2).astype(np.float32)
        got = m.forward(torch.from_numpy(X).cuda()).cpu().numpy()
        for b in range(X.shape[0]):
            want = O.mlp_forward_f32(q, X[b])
            assert np.array_equal(got[b], want), b
            _, _, o64 = O.mlp_forward_f64(q.astype(np.float64), X[b].astype(np.float64))
            assert np.all(np.abs(got[b] - o64) <= 1e-3 * np.maximum(np.abs(o64), 1e-2))
    m.close()


@pytest.mark.parametrize("B", [1, 64, 300])
def test_gradient_against_binary64(B):
    m = dd.Mlp()
    p = random_params(20 + B)
    m.set_params(p)
    q = evaluated(p).astype(np.float64)
    rng = np.random.default_rng(B)
    X = (rng.random((B, 128)) * 2).astype(np.float32)
    u = rng.uniform(0.0, 0.35, B).astype(np.float32)
    g, loss = m.grad(torch.from_numpy(X).cuda(), torch.from_numpy(u).cuda())
    g = g.cpu().numpy().astype(np.float64)
    want_loss, want = O.mlp_loss_f64(q, X.astype(np.float64), u.astype(np.float64))
    assert abs(float(loss.item()) - want_loss) <= 1e-3 * abs(want_loss)
    o = O.OFFSETS
    for a, b in (("W1", "b1"), ("b1", "W2"), ("W2", "b2"), ("b2", "W3"), ("W3", "b3"), ("b3", None)):
        sl = slice(o[a], o[b] if b else None)
        err = np.linalg.norm(g[sl] - want[sl]) / max(np.linalg.norm(want[sl]), 1e-12)
        assert err <= 1e-2, (a, err)
    m.close()


def test_training_lowers_the_loss_and_checkpoints(tmp_path):
    rng = np.random.default_rng(6)
    X = torch.from_numpy((rng.random((256, 128)) * 2).astype(np.float32)).cuda()
    u = torch.from_numpy(rng.uniform(0.0, 0.3, 256).astype(np.float32)).cuda()
    m = dd.Mlp(seed=7)
    _, l0 = m.grad(X, u)
    loss = torch.empty(1, device="cuda")
    for _ in range(200):
        m.train_step(X, u, 1e-3, loss)
    _, l1 = m.grad(X, u)
    assert float(l1.item()) < float(l0.item()) - 0.5
    path = os.path.join(str(tmp_path), "m.bin")
    m.save(path)
    m2 = dd.Mlp(seed=99, path=path)
    assert np.array_equal(m2.get_params(), m.get_params())
    assert torch.equal(m2.forward(X), m.forward(X))
    with open(path, "r+b") as f:                      # a damaged header is refused
        f.write(b"XXXX")
    with pytest.raises(dd.DDError):
        m2.load(path)
    m.close()
    m2.close()


# ------------------------------------------------------ warm-started search

def assert_same(a, b, trace=False):
    for k in KEYS:
        assert a[k] == b[k], (k, a[k], b[k])
    if trace:
        assert a["trace"] == b["trace"]


@pytest.mark.parametrize("pop_k,host_loop", [(1, 0), (16, 0), (4, 1)])
def test_given_warm_start_matches_oracle(pop_k, host_loop):
    w = window_config1()
    win = O.Window.of(w)
    ctx = dd.Context(w.W, w.H, w.foe_x, w.foe_y, pop_k=pop_k, host_loop=host_loop)
    ev = dd.Events.of(w, device="cuda")
    for guess in ((0.2, 0.02), (-0.6, 0.125), (1.7, 0.25), (-1.0, 0.5), (0.0, 4.0), (0.19, 2.0 ** -14)):
        r = ctx.solve(ev, -1.0, 1.0, 1e-4, 0.0, trace_cap=4096, warm=guess)
        want = O.solve(win, -1.0, 1.0, 1e-4, 0.0, pop_k, trace_cap=4096, warm=guess)
        assert_same(r, want, trace=True)
        d0 = float(np.float32(min(max(np.float32(guess[0]), -1.0), 1.0)))
        assert r["D_warm"] == d0 and r["w_warm"] == np.float32(guess[1])
    ctx.close()


def oracle_model_solve(win, p_eval, D_lo, D_hi, tol, gamma, K):
    f, _ = O.features(win)
    u, l = O.mlp_forward_f32(p_eval, f)
    guess = O.warm_map(float(u), float(l), win.c.tau)
    return O.solve(win, D_lo, D_hi, tol, gamma, K, warm=guess), guess


def test_model_warm_start_matches_oracle_end_to_end():
    p = random_params(31)
    q = evaluated(p)
    m = dd.Mlp()
    m.set_params(p)
    ws = [window_config1(), window_config1(seed=1001), window_config1(seed=1002)]
    ctx = dd.Context(346, 260, 173.0, 130.0, pop_k=8)
    ctx.set_warm_model(m)
    for w in ws:
        win = O.Window.of(w)
        want, guess = oracle_model_solve(win, q, -1.0, 1.0, 1e-4, 0.0, 8)
        r = ctx.solve(dd.Events.of(w, device="cuda"), warm="model")
        assert_same(r, want)
        assert (r["D_warm"], r["w_warm"]) == (np.float32(min(max(guess[0], -1.0), 1.0)), np.float32(guess[1]))
    ctx.close()
    m.close()


def test_batch_with_mixed_warm_starts():
    p = random_params(41)
    q = evaluated(p)
    m = dd.Mlp()
    m.set_params(p)
    ws = [make_window(640, 480, 320.0, 240.0, 7000 + 3000 * i, 200 + 50 * i, 2000, 0.1 + 0.1 * i, 0.3, 700 + i)
          for i in range(6)]
    warms = [None, "model", (0.25, 0.03), "model", None, (5.0, 0.1)]
    params = [(-1.0, 1.0, 1e-4, 0.0, wm) for wm in warms]
    ctx = dd.Context(640, 480, 320.0, 240.0, pop_k=8)
    ctx.set_warm_model(m)
    rc, res = ctx.solve_batch([dd.Events.of(w, device="cuda" if i % 2 else None) for i, w in enumerate(ws)],
                              params)
    assert rc == dd.DD_OK
    for w, wm, r in zip(ws, warms, res):
        win = O.Window.of(w)
        if wm == "model":
            want, _ = oracle_model_solve(win, q, -1.0, 1.0, 1e-4, 0.0, 8)
        else:
            want = O.solve(win, -1.0, 1.0, 1e-4, 0.0, 8, warm=wm)
        assert_same(r, want)
    ctx.close()
    m.close()


def test_serving_with_warm_starts_matches_solo():
    p = random_params(51)
    m = dd.Mlp()
    m.set_params(p)
    ctx = dd.Context(1280, 720, 640.0, 360.0, pop_k=8)
    ctx.set_warm_model(m)
    ws = [serve_config5(s, 30 + 40 * k, n_scale=0.02) for s in range(2) for k in range(3)]
    warms = ["model", None, (0.06, 0.01), "model", "model", None]
    srv = dd.Server(ctx, max_slots=3, max_events=1 << 16)
    params = [(-1.0, 2.0, 1e-4, 0.0, wm) for wm in warms]
    tickets = [srv.submit(dd.Events.of(w, device="cuda"), pp) for w, pp in zip(ws, params)]
    got = [srv.wait(t) for t in tickets]
    srv.stop()
    for w, pp, r in zip(ws, params, got):
        one = ctx.solve(dd.Events.of(w, device="cuda"), *pp[:4], warm=pp[4])
        assert_same(r, one)
        assert (r["D_warm"], r["w_warm"]) == (one["D_warm"], one["w_warm"])
    ctx.close()
    m.close()


def test_warm_start_argument_errors():
    w = window_config1()
    ctx = dd.Context(w.W, w.H, w.foe_x, w.foe_y)
    ev = dd.Events.of(w, device="cuda")
    with pytest.raises(dd.DDError) as e:                 # no model set
        ctx.solve(ev, warm="model")
    assert e.value.status == dd.DD_ERR_ARG
    for bad in ((0.1, 0.0), (0.1, -1.0), (float("nan"), 0.1), (0.1, float("inf"))):
        with pytest.raises(dd.DDError) as e:
            ctx.solve(ev, warm=bad)
        assert e.value.status == dd.DD_ERR_ARG
    r = ctx.solve(ev)
    assert r["D_warm"] == 0.0 and r["w_warm"] == 0.0
    ctx.close()


def test_trained_model_gains_over_the_plain_search():
    # The committed model (trained on 200k windows labelled by the exact
    # solver) against Algorithm 1 from the centre on held-out windows: fewer
    # rounds and nodes in total, and every pair of certificates consistent
    # (each K_hat within the other's certified gap; identical where both are
    # exact).
    from paper_2209_13168_gb300 import warm_start
    from synth.descent import WARM_EVAL_SEED
    from synth.gpu import make_window_gpu
    specs = warm_start.window_specs(128, WARM_EVAL_SEED + 50_000)
    ws = [make_window_gpu(s) for s in specs]
    evs = [dd.Events.of(w) for w in ws]
    ctx = dd.Context(640, 480, 320.0, 240.0, pop_k=16, band_rows=38, threads=512)
    m = dd.Mlp(path=warm_start.DEFAULT_MODEL)
    ctx.set_warm_model(m)
    rc0, plain = ctx.solve_batch(evs, [(-1.0, 1.0, 1e-4, 0.0)] * len(evs))
    rc1, learned = ctx.solve_batch(evs, [(-1.0, 1.0, 1e-4, 0.0, "model")] * len(evs))
    assert rc0 == dd.DD_OK and rc1 == dd.DD_OK
    for a, b in zip(plain, learned):
        assert a["K_hat"] <= b["K_hat"] + b["gap_K"] and b["K_hat"] <= a["K_hat"] + a["gap_K"]
        if a["gap_K"] == 0 and b["gap_K"] == 0:
            assert a["K_hat"] == b["K_hat"]
    rounds = (sum(r["rounds"] for r in plain), sum(r["rounds"] for r in learned))
    nodes = (sum(r["nodes_expanded"] for r in plain), sum(r["nodes_expanded"] for r in learned))
    assert rounds[1] < 0.95 * rounds[0], rounds
    assert nodes[1] < nodes[0], nodes
    # the guesses are informative: most lie within their half-width of D*
    inside = sum(abs(b["D_warm"] - a["D_star"]) <= b["w_warm"] for a, b in zip(plain, learned))
    assert inside >= 0.8 * len(ws)
    ctx.close()
    m.close()


def test_training_labels_match_the_oracle():
    # The training targets are the exact batch solver's D* (u* = D* tau): a
    # sample of training windows (the three smallest of the first 64) is
    # re-solved by the oracle with the same pop width.
    from paper_2209_13168_gb300 import warm_start
    from synth.descent import WARM_TRAIN_SEED
    specs = warm_start.window_specs(64, WARM_TRAIN_SEED)
    pick = sorted(range(64), key=lambda i: specs[i][4] + specs[i][6])[:3]
    ctx = warm_start.context()
    _, u, D, _ = warm_start.label(ctx, [specs[i] for i in pick], log=None)
    u = u.cpu().numpy()
    for j, i in enumerate(pick):
        w = make_window(*specs[i])
        want = O.solve(O.Window.of(w), *warm_start.PARAMS, ctx.cfg.pop_k)
        assert float(D[j]) == want["D_star"]
        assert u[j] == np.float32(np.float64(want["D_star"]) * np.float64(np.float32(w.tau)))
    ctx.close()
