"""The GPU window generator reproduces the numpy generator event for event."""
import numpy as np
import pytest

from synth import make_window
from synth.descent import batch_params3, batch_spec3, serve_spec5

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

from synth.gpu import make_window_gpu  # noqa: E402


def as_sorted(x, y, t, p=None):
    cols = [np.asarray(t, np.float64), np.asarray(x, np.float64), np.asarray(y, np.float64)]
    if p is not None:
        cols.append(np.asarray(p, np.float64))
    a = np.stack(cols, axis=1)
    return a[np.lexsort(tuple(a[:, k] for k in range(a.shape[1] - 1, -1, -1)))]


@pytest.mark.parametrize("spec", [
    (346, 260, 173.0, 130.0, 3000, 150, 1000, 0.2, 0.5, 1000),
    (640, 480, 320.0, 240.0, 70000, 2000, 30000, 0.35, 0.3, 2000),
    (97, 61, 48.5, 30.0, 900, 45, 300, -0.45, 0.35, 9),
    serve_spec5(2, 150, n_scale=0.05),
])
def test_gpu_generator_matches_numpy(spec):
    w = make_window(*spec)
    g = make_window_gpu(spec)
    assert g.n == w.n
    a = as_sorted(w.x, w.y, w.t)
    b = as_sorted(g.x.cpu().numpy(), g.y.cpu().numpy(), g.t.cpu().numpy())
    assert np.array_equal(a, b)


def test_gpu_generator_batch_windows():
    params = batch_params3()
    for i in (0, 5, 77):
        spec = batch_spec3(i, params)
        w = make_window(*spec)
        g = make_window_gpu(spec)
        assert np.array_equal(as_sorted(w.x, w.y, w.t),
                              as_sorted(g.x.cpu().numpy(), g.y.cpu().numpy(), g.t.cpu().numpy()))


@pytest.mark.parametrize("spec", [
    (346, 260, 173.0, 130.0, 3000, 150, 1000, 0.2, 0.5, 1000),
    (97, 61, 48.5, 30.0, 900, 45, 300, -0.45, 0.35, 9),
])
def test_gpu_generator_polarities(spec):
    # (t, x, y, p) as a multiset: the polarity of every event as numpy draws it
    w = make_window(*spec)
    g = make_window_gpu(spec, polarity=True)
    assert np.array_equal(as_sorted(w.x, w.y, w.t, w.p),
                          as_sorted(g.x.cpu().numpy(), g.y.cpu().numpy(), g.t.cpu().numpy(), g.p.cpu().numpy()))
    assert set(np.unique(w.p)) == {-1, 1}
