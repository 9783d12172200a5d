"""The start-of-window warp (reference time 0) on the GPU against the oracle:
images, keys and searches bit for bit, as for the paper's warp."""
import numpy as np
import pytest

import oracle as O
from synth import window_config1, window_config2
from synth.descent import batch_params3, batch_window3

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2209_13168_gb300 as dd  # noqa: E402

KEYS = ("D_star", "D_end", "K_hat", "gap_K", "nodes_expanded", "point_evals", "bound_evals", "cell_increments",
        "bound_increments", "rounds", "max_queue")


@pytest.mark.parametrize("make", [window_config1, window_config2])
def test_images_at_t_ref_0(make):
    w = make()
    win = O.Window.of(w, t_ref=0.0)
    ctx = dd.Context(w.W, w.H, w.foe_x, w.foe_y, warp_to_start=1)
    ev = dd.Events.of(w, device="cuda")
    Ds = np.array([-1.0, -0.2, 0.0, 0.2, 0.35, 1.0], np.float32)
    K, S, N, img = ctx.contrast(ev, Ds, want_iwe=True)
    for j, D in enumerate(Ds):
        k, s, n, im = O.contrast(win, float(D), want_iwe=True)
        assert (K[j], int(S[j]), int(N[j])) == (k, s, n)
        assert np.array_equal(img[j], im)
    lo = np.array([-1.0, 0.1, 0.3], np.float32)
    hi = np.array([1.0, 0.2, 0.3001], np.float32)
    Kb, Sb, Nb, _ = ctx.bound(ev, lo, hi)
    for j in range(3):
        assert (Kb[j], int(Sb[j]), int(Nb[j])) == O.bound(win, float(lo[j]), float(hi[j]))[:3]
    ctx.close()


@pytest.mark.parametrize("pop_k", [1, 16])
def test_solve_at_t_ref_0(pop_k):
    for w in (window_config1(), window_config2()):
        ctx = dd.Context(w.W, w.H, w.foe_x, w.foe_y, pop_k=pop_k, warp_to_start=1)
        got = ctx.solve(dd.Events.of(w, device="cuda"), trace_cap=4096)
        want = O.solve(O.Window.of(w, t_ref=0.0), -1.0, 1.0, 1e-4, 0.0, pop_k, trace_cap=4096)
        for k in KEYS:
            assert got[k] == want[k], (k, got[k], want[k])
        assert got["trace"] == want["trace"]
        ctx.close()


def test_batch_at_t_ref_0():
    params = batch_params3()
    ws = [batch_window3(i, params) for i in (142, 68, 62, 228)]        # the smallest windows
    ctx = dd.Context(640, 480, 320.0, 240.0, pop_k=8, warp_to_start=1)
    rc, res = ctx.solve_batch([dd.Events.of(w, device="cuda") for w in ws])
    assert rc == dd.DD_OK
    for w, r in zip(ws, res):
        want = O.solve(O.Window.of(w, t_ref=0.0), -1.0, 1.0, 1e-4, 0.0, 8)
        for k in KEYS:
            assert r[k] == want[k], k
    ctx.close()
