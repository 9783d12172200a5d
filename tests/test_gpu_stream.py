"""The stream-wise estimation (Sec. 4.4) on the GPU: a continuous descent
stream solved window by window must give, for every window, the oracle's
result on the same slice of the stream, and the time to contact 1/D_end."""
import numpy as np
import pytest

import oracle as O
from synth.descent import stream_events5

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2209_13168_gb300 as dd  # noqa: E402

KEYS = ("D_star", "D_end", "K_hat", "gap_K", "nodes_expanded", "point_evals", "bound_evals", "cell_increments",
        "bound_increments", "rounds")
PARAMS = (-1.0, 2.0, 1e-4, 0.0)


def numpy_slice(t, t0, tau):
    """The events whose binary32 t - t0 lies in [0, tau] (t sorted)."""
    d = (t - np.float32(t0)).astype(np.float32)
    idx = np.nonzero((d >= 0) & (d <= np.float32(tau)))[0]
    return (int(idx[0]) if idx.size else int(np.searchsorted(d, 0.0))), idx.size


@pytest.mark.parametrize("device", [None, "cuda"])
def test_stream_windows_match_oracle(device):
    x, y, t = stream_events5(0, 100, 112, n_scale=0.02)          # 1.2 s of the descent from t = 10 s
    ev = dd.Events(x, y, t, 0.0, 1.0) if device is None else dd.Events(
        torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), torch.from_numpy(t).cuda(), 0.0, 1.0)
    ctx = dd.Context(1280, 720, 640.0, 360.0, pop_k=8)
    n_win, tau, hop = 10, np.float32(0.2), 0.1
    rc, res, ttc, first = ctx.stream_solve(ev, 10.0, float(tau), hop, n_win, PARAMS)
    assert rc == dd.DD_OK
    for k in range(n_win):
        t0 = np.float32(10.0 + hop * k)
        f, n = numpy_slice(t, t0, tau)
        assert first[k] == f
        win = O.Window(1280, 720, 640.0, 360.0, x[f:f + n], y[f:f + n], t[f:f + n], float(t0), float(tau))
        want = O.solve(win, *PARAMS, 8)
        for key in KEYS:
            assert res[k][key] == want[key], (k, key)
        assert ttc[k] == np.float32(1.0) / np.float32(res[k]["D_end"])
        # the true divergence at the window's end is 1/(20 - t0 - tau)
        assert abs(res[k]["D_end"] - 1.0 / (20.0 - float(t0) - float(tau))) < 0.05
    ctx.close()


def test_stream_edges_and_errors():
    x, y, t = stream_events5(1, 50, 53, n_scale=0.01)
    ev = dd.Events(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), torch.from_numpy(t).cuda(), 0.0, 1.0)
    ctx = dd.Context(1280, 720, 640.0, 360.0, pop_k=4)
    # windows past the end of the stream are empty: no events, zero contrast
    rc, res, ttc, first = ctx.stream_solve(ev, 5.0, 0.2, 0.1, 5, PARAMS)
    assert rc == dd.DD_OK
    assert res[4]["K_hat"] == 0 and first[4] == x.size
    for bad in ((0.0, 0.1), (0.2, 0.0), (-0.2, 0.1)):
        with pytest.raises(dd.DDError):
            ctx.stream_solve(ev, 5.0, bad[0], bad[1], 3, PARAMS)
    ctx.close()
