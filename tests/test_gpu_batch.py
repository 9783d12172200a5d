"""GPU parity of the batched solver: many windows, one launch sequence.

Each window's result must be bit-identical to the oracle's Algorithm 1 on
that window alone (same pop width), and to the single-window GPU solve.
"""
import numpy as np
import pytest

import oracle as O
from synth import make_window
from synth.descent import batch_params3, batch_window3

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2209_13168_gb300 as dd  # noqa: E402

KEYS = ("D_star", "D_end", "K_hat", "gap_K", "nodes_expanded", "point_evals", "bound_evals", "event_warps",
        "cell_increments", "bound_increments", "rounds", "max_queue")


def small_batch(n, seed=0):
    rng = np.random.default_rng(seed)
    ws = []
    for i in range(n):
        N = int(rng.integers(200, 6000))
        noise = int(N * rng.uniform(0.1, 0.4))
        D = float(rng.uniform(0.05, 0.8))
        tau = float(rng.uniform(0.1, 0.5))
        ws.append(make_window(160, 120, 80.0, 60.0, N - noise, max(1, (N - noise) // 35), noise, D, tau,
                              seed=100 + i))
    return ws


@pytest.mark.parametrize("pop_k,host_loop", [(1, 0), (8, 0), (8, 1)])
def test_batch_matches_oracle_per_window(pop_k, host_loop):
    ws = small_batch(12)
    ctx = dd.Context(160, 120, 80.0, 60.0, pop_k=pop_k, host_loop=host_loop)
    evs = [dd.Events.of(w, device="cuda") for w in ws]
    rc, res = ctx.solve_batch(evs)
    assert rc == dd.DD_OK
    for w, r in zip(ws, res):
        want = O.solve(O.Window.of(w), -1.0, 1.0, 1e-4, 0.0, pop_k)
        for k in KEYS:
            assert r[k] == want[k], (k, r[k], want[k])
        assert r["status"] == dd.DD_OK
    # the same windows one by one
    for ev, r in zip(evs[:4], res[:4]):
        one = ctx.solve(ev)
        for k in KEYS:
            assert one[k] == r[k], k
    ctx.close()


def test_batch_params_per_window_and_mixed_inputs():
    ws = small_batch(5, seed=3)
    ctx = dd.Context(160, 120, 80.0, 60.0, pop_k=4)
    evs = [dd.Events.of(w, device="cuda" if i % 2 else None) for i, w in enumerate(ws)]
    params = [(-1.0, 1.0, 1e-4, 0.0), (0.0, 1.0, 1e-3, 0.0), (-0.5, 0.9, 1e-4, 0.01), (0.1, 0.5, 1e-5, 0.0),
              (-1.0, 1.0, 1e-4, 0.0)]
    rc, res = ctx.solve_batch(evs, params)
    assert rc == dd.DD_OK
    for w, p, r in zip(ws, params, res):
        want = O.solve(O.Window.of(w), p[0], p[1], p[2], p[3], 4)
        for k in KEYS:
            assert r[k] == want[k], (k, p)
    ctx.close()


def test_batch_reports_a_malformed_window_and_solves_the_others():
    ws = small_batch(4, seed=5)
    ws[2].t[7] = np.float32(ws[2].tau * 2.0)         # outside its window
    ctx = dd.Context(160, 120, 80.0, 60.0, pop_k=4)
    evs = [dd.Events.of(w, device="cuda") for w in ws]
    rc, res = ctx.solve_batch(evs)
    assert rc == dd.DD_ERR_ARG and res[2]["status"] == dd.DD_ERR_ARG
    for i in (0, 1, 3):
        want = O.solve(O.Window.of(ws[i]), -1.0, 1.0, 1e-4, 0.0, 4)
        assert res[i]["status"] == dd.DD_OK
        assert res[i]["K_hat"] == want["K_hat"] and res[i]["nodes_expanded"] == want["nodes_expanded"]
    # the context keeps working
    rc, res2 = ctx.solve_batch([evs[0], evs[1]])
    assert rc == dd.DD_OK and res2[0]["K_hat"] == res[0]["K_hat"]
    ctx.close()


def test_uneven_256_window_batch_sampled_against_oracle():
    # The 256-window workload (640x480, N log-uniform in [5k, 200k]) in the
    # configuration bench.py times (the autotuned batch knobs): every 17th
    # window against its single-window GPU solve, a sample against the oracle.
    params = batch_params3()
    ws = [batch_window3(i, params) for i in range(256)]
    ctx = dd.Context.tuned(640, 480, 320.0, 240.0, sum(w.n for w in ws) / len(ws), mode="batch")
    pop_k = ctx.cfg.pop_k
    evs = [dd.Events.of(w, device="cuda") for w in ws]
    rc, res = ctx.solve_batch(evs)
    assert rc == dd.DD_OK
    for i in range(0, 256, 17):
        one = ctx.solve(evs[i])
        for k in KEYS:
            assert one[k] == res[i][k], (i, k)
    order = np.argsort(params[0])
    for i in list(order[:3]) + [int(order[128])]:
        want = O.solve(O.Window.of(ws[i]), -1.0, 1.0, 1e-4, 0.0, pop_k)
        for k in KEYS:
            assert res[i][k] == want[k], (i, k)
    for i in range(256):
        assert abs(res[i]["D_star"] - params[1][i]) < 0.05, i
    ctx.close()
