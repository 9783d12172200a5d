"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Integer results (IWE counts, sums of squares, keys, node counts, traces) must
be bit-identical; D* must be the same binary32 value.  Inputs are the seeded
synthetic windows of synth/ at the workload sizes, plus ragged and degenerate
cases.
"""
import numpy as np
import pytest

import oracle as O
from synth import make_window, window_config1, window_config2, serve_config5
from synth.descent import batch_params3, batch_window3

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2209_13168_gb300 as dd  # noqa: E402


@pytest.fixture(scope="module")
def c1():
    return window_config1()


@pytest.fixture(scope="module")
def c2():
    return window_config2()


def ctx_for(w, **kw):
    return dd.Context(w.W, w.H, w.foe_x, w.foe_y, **kw)


def check_contrast(w, Ds, want_iwe, **kw):
    kw.pop("host_loop", None)
    ctx = ctx_for(w, **kw)
    win = O.Window.of(w)
    for dev in (None, "cuda"):
        ev = dd.Events.of(w, device=dev)
        K, S, N, img = ctx.contrast(ev, Ds, want_iwe=want_iwe)
        for j, D in enumerate(Ds):
            k, s, n, im = O.contrast(win, float(D), want_iwe=want_iwe)
            assert (K[j], int(S[j]), int(N[j])) == (k, s, n), (D, dev)
            if want_iwe:
                assert np.array_equal(img[j], im), D
    ctx.close()


def check_bound(w, lo, hi, want_iwe, **kw):
    kw.pop("host_loop", None)
    ctx = ctx_for(w, **kw)
    win = O.Window.of(w)
    ev = dd.Events.of(w, device="cuda")
    K, S, N, img = ctx.bound(ev, lo, hi, want_iwe=want_iwe)
    for j in range(len(lo)):
        k, s, n, im = O.bound(win, float(lo[j]), float(hi[j]), want_iwe=want_iwe)
        assert (K[j], int(S[j]), int(N[j])) == (k, s, n), (lo[j], hi[j])
        if want_iwe:
            assert np.array_equal(img[j], im), (lo[j], hi[j])
    ctx.close()


def intervals(rng, n, tau, lo=-1.0, hi=1.0):
    a = rng.uniform(lo, hi, n)
    width = 10 ** rng.uniform(-4.5, np.log10(hi - lo), n)
    b = np.minimum(a + width, min(hi, 0.75 / tau))
    a, b = a.astype(np.float32), b.astype(np.float32)
    keep = a < b
    return a[keep], b[keep]


def check_solve(w, pop_k, D_lo=-1.0, D_hi=1.0, tol=1e-4, gamma=0.0, trace=True, **kw):
    ctx = ctx_for(w, pop_k=pop_k, **kw)
    ev = dd.Events.of(w, device="cuda")
    got = ctx.solve(ev, D_lo, D_hi, tol, gamma, trace_cap=4096 if trace else 0)
    want = O.solve(O.Window.of(w), D_lo, D_hi, tol, gamma, pop_k, trace_cap=4096 if trace else 0)
    for k in ("D_star", "D_end", "K_hat", "gap_K", "nodes_expanded", "point_evals", "bound_evals",
              "event_warps", "cell_increments", "bound_increments", "rounds", "max_queue"):
        assert got[k] == want[k], (k, got[k], want[k])
    assert got["contrast"] == want["contrast"] and got["bound_gap"] == want["bound_gap"]
    if trace:
        assert got["trace_len"] == want["trace_len"]
        assert got["trace"] == want["trace"]
    ctx.close()
    return got


# ---------------------------------------------------------------- contrast

def test_contrast_iwe_config1(c1):
    Ds = np.concatenate([[0.0, 0.2, -1.0, 1.0], np.linspace(-1, 1, 60)]).astype(np.float32)
    check_contrast(c1, Ds, want_iwe=True)


def test_contrast_keys_config2(c2):
    rng = np.random.default_rng(3)
    Ds = np.concatenate([[0.0, 0.35, -1.0, 1.0], rng.uniform(-1, 1, 150), 0.35 + rng.normal(0, 0.01, 50)])
    check_contrast(c2, Ds.astype(np.float32), want_iwe=False)
    check_contrast(c2, np.array([0.0, 0.35, -0.6, 0.9], np.float32), want_iwe=True)


# ------------------------------------------------------------------- bound

def test_bound_iwe_config1(c1):
    rng = np.random.default_rng(5)
    lo, hi = intervals(rng, 40, c1.tau)
    lo = np.concatenate([[-1.0, 0.0, 0.19], lo]).astype(np.float32)
    hi = np.concatenate([[1.0, 0.5, 0.2001], hi]).astype(np.float32)
    check_bound(c1, lo, hi, want_iwe=True)


def test_bound_keys_config2(c2):
    rng = np.random.default_rng(6)
    lo, hi = intervals(rng, 60, c2.tau)
    check_bound(c2, lo, hi, want_iwe=False)
    check_bound(c2, np.array([-1.0, 0.3], np.float32), np.array([1.0, 0.4], np.float32), want_iwe=True)


# ------------------------------------------------------------------- solve

@pytest.mark.parametrize("pop_k", [1, 4, 16])
@pytest.mark.parametrize("host_loop", [0, 1])
def test_solve_config1(c1, pop_k, host_loop):
    check_solve(c1, pop_k, host_loop=host_loop)


@pytest.mark.parametrize("pop_k", [1, 16])
def test_solve_config2(c2, pop_k):
    r = check_solve(c2, pop_k)
    assert abs(r["D_star"] - 0.35) <= 0.02


def test_solve_config2_in_the_benchmark_configuration(c2):
    # The context bench.py times: the autotuned knobs for this geometry and
    # size (pop width, band rows, threads, split cap), solved as one graph.
    ctx = dd.Context.tuned(c2.W, c2.H, c2.foe_x, c2.foe_y, c2.n, mode="single")
    pop_k = ctx.cfg.pop_k
    ev = dd.Events.of(c2, device="cuda")
    got = ctx.solve(ev, -1.0, 1.0, 1e-4, 0.0, trace_cap=4096)
    plain = ctx.solve(ev)                         # the graph path, as timed
    want = O.solve(O.Window.of(c2), -1.0, 1.0, 1e-4, 0.0, pop_k, trace_cap=4096)
    for k in ("D_star", "D_end", "K_hat", "gap_K", "nodes_expanded", "point_evals", "bound_evals",
              "event_warps", "cell_increments", "bound_increments", "rounds", "max_queue"):
        assert got[k] == want[k], (k, got[k], want[k])
        assert plain[k] == want[k], (k, plain[k], want[k])
    assert got["trace"] == want["trace"]
    ctx.close()


def test_solve_with_gamma_and_narrow_range(c1):
    check_solve(c1, 1, gamma=0.025)
    check_solve(c1, 2, D_lo=0.15, D_hi=0.25, tol=1e-5)


def test_solve_repeat_is_identical(c1, c2):
    # The same context across windows of different sizes (buffers regrow and
    # the solve graph is rebuilt) and with and without a trace.
    ctx = ctx_for(c1, pop_k=4)
    ev1 = dd.Events.of(c1, device="cuda")
    a = ctx.solve(ev1)
    b = ctx.solve(ev1, trace_cap=10)
    c = ctx.solve(ev1)
    for k in a:
        assert a[k] == b[k] == c[k], k
    ctx.close()
    ctx = ctx_for(c2, pop_k=8)
    small = make_window(640, 480, 320.0, 240.0, 7000, 200, 3000, 0.35, 0.3, seed=21)
    r_small = ctx.solve(dd.Events.of(small, device="cuda"))
    r_big = ctx.solve(dd.Events.of(c2, device="cuda"))
    r_small2 = ctx.solve(dd.Events.of(small, device="cuda"))
    assert r_small == r_small2
    assert r_big["K_hat"] == O.solve(O.Window.of(c2), -1.0, 1.0, 1e-4, 0.0, 8)["K_hat"]
    ctx.close()


# ------------------------------------------------------------ edge cases

def test_ragged_tiles_and_thread_counts():
    w = make_window(97, 61, 48.5, 30.0, 900, 45, 300, 0.45, 0.35, seed=9)
    rng = np.random.default_rng(1)
    Ds = rng.uniform(-1, 1, 20).astype(np.float32)
    lo, hi = intervals(rng, 12, w.tau)
    for kw in ({}, {"band_rows": 1}, {"band_rows": 7, "threads": 64}, {"band_rows": 61, "threads": 512},
               {"band_rows": 5, "threads": 96, "host_loop": 1}):
        check_contrast(w, Ds, want_iwe=True, **kw)
        check_bound(w, lo, hi, want_iwe=True, **kw)
        check_solve(w, 3, trace=True, **kw)


@pytest.mark.parametrize("band_rows", [1, 3, 16])
def test_band_candidates_at_the_ends_of_the_domain(band_rows):
    # Which events a row band reads is decided from binary32 bounds with
    # margins: at the ends of the domain (D tau from -50 to 0.745), with a
    # non-integer FOE and dense events, every image must still equal the
    # oracle's.
    w = make_window(200, 150, 99.37, 74.81, 16000, 800, 4000, 0.6, 0.5, 77)
    tau = w.tau
    Ds = np.array([-100.0, -10.0, -1.0, 0.0, 0.5, 1.0, 1.4, 0.745 / tau], np.float32)
    lo = np.array([-100.0, -2.0, 1.2, 1.48, 0.0], np.float32)
    hi = np.array([-99.0, 1.49, 1.49, 0.745 / tau, 1e-3], np.float32)
    for want_iwe in (True, False):            # images copied out, or only keys
        check_contrast(w, Ds, want_iwe, band_rows=band_rows)
        check_bound(w, lo, hi, want_iwe, band_rows=band_rows)


def test_degenerate_windows():
    empty = make_window(40, 30, 20.0, 15.0, 0, 1, 0, 0.3, 0.5, seed=1)
    check_solve(empty, 1)
    check_contrast(empty, np.array([0.0, 0.5], np.float32), want_iwe=True)
    one = make_window(40, 30, 20.0, 15.0, 1, 1, 0, 0.3, 0.5, seed=2)
    check_solve(one, 1)
    # all events on the FOE pixel
    n = 50
    foe = dict(W=33, H=21, foe_x=16.0, foe_y=10.0)
    w = make_window(33, 21, 16.0, 10.0, 0, 1, n, 0.3, 0.4, seed=3)
    w.x[:] = 16
    w.y[:] = 10
    check_solve(w, 1)
    check_bound(w, np.array([-1.0], np.float32), np.array([1.5], np.float32), want_iwe=True)
    # all events at t = tau: constant contrast, no expansion
    w = make_window(64, 48, 32.0, 24.0, 500, 25, 100, 0.3, 0.5, seed=4)
    w.t[:] = np.float32(0.5)
    r = check_solve(w, 1, D_hi=1.5)
    assert r["nodes_expanded"] == 0
    del foe


def test_time_offset_and_host_pointers():
    w = make_window(120, 90, 60.0, 45.0, 2000, 80, 500, 0.25, 0.4, seed=11, t0=3.25)
    check_contrast(w, np.linspace(-1, 1, 9).astype(np.float32), want_iwe=True)
    ctx = ctx_for(w)
    a = ctx.solve(dd.Events.of(w))
    b = ctx.solve(dd.Events.of(w, device="cuda"))
    assert a == b
    want = O.solve(O.Window.of(w), -1.0, 1.0, 1e-4, 0.0, 1)
    assert a["K_hat"] == want["K_hat"] and a["nodes_expanded"] == want["nodes_expanded"]
    ctx.close()


# ------------------------------------------------------- large workloads

def test_sampled_parity_large_windows():
    # The largest single windows of the workloads: a 200k-event window of the
    # uneven batch and a late 1280x720 serving window, at sampled hypotheses.
    params = batch_params3()
    i = int(np.argmax(params[0]))
    wb = batch_window3(i, params)
    check_contrast(wb, np.array([0.0, float(params[1][i]), -0.7, 0.9], np.float32), want_iwe=False)
    ws = serve_config5(0, 180, n_scale=0.5)
    check_contrast(ws, np.array([0.0, ws.D_true, 1.9], np.float32), want_iwe=False)
    lo = np.array([-1.0, ws.D_true - 0.01], np.float32)
    hi = np.array([2.0, ws.D_true + 0.01], np.float32)
    check_bound(ws, lo, hi, want_iwe=False)


# ------------------------------------------------------------------ errors

def test_errors_are_reported_not_faulted(c1):
    ctx = ctx_for(c1)
    ev = dd.Events.of(c1, device="cuda")
    with pytest.raises(dd.DDError) as e:
        ctx.solve(ev, -1.0, 1.6)              # D_hi * tau > 3/4
    assert e.value.status == dd.DD_ERR_ARG
    bad = make_window(40, 30, 20.0, 15.0, 20, 2, 5, 0.3, 0.5, seed=5)
    bad.t[3] = np.float32(0.75)               # outside [t0, t0 + tau]
    with pytest.raises(dd.DDError) as e:
        ctx.solve(dd.Events.of(bad))
    assert e.value.status == dd.DD_ERR_ARG
    bctx = ctx_for(bad)
    for dev in ("cuda",):
        with pytest.raises(dd.DDError) as e:
            bctx.solve(dd.Events.of(bad, device=dev))
        assert e.value.status == dd.DD_ERR_ARG
        with pytest.raises(dd.DDError) as e:
            bctx.contrast(dd.Events.of(bad, device=dev), [0.1])
        assert e.value.status == dd.DD_ERR_ARG
    bctx.close()
    small = ctx_for(c1, queue_capacity=4)
    with pytest.raises(dd.DDError) as e:
        small.solve(ev)
    assert e.value.status == dd.DD_ERR_QUEUE_OVERFLOW
    small.close()
    short = ctx_for(c1, max_rounds=3)
    with pytest.raises(dd.DDError) as e:
        short.solve(ev)
    assert e.value.status == dd.DD_ERR_TIMEOUT
    short.close()
    # the context is still usable after errors
    r = ctx.solve(ev)
    assert r["K_hat"] == O.solve(O.Window.of(c1), -1.0, 1.0, 1e-4, 0.0, 1)["K_hat"]
    ctx.close()
