"""Per-solve JSONL log and the image helper on the GPU."""
import json

import numpy as np
import pytest

import oracle as O
from synth import make_window, window_config1

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

import paper_2209_13168_gb300 as dd  # noqa: E402


def test_solve_log_has_one_line_per_window(tmp_path):
    w = window_config1()
    ctx = dd.Context(w.W, w.H, w.foe_x, w.foe_y, pop_k=4)
    log = tmp_path / "solves.jsonl"
    ctx.set_log(str(log))
    ev = dd.Events.of(w, device="cuda")
    r1 = ctx.solve(ev)
    rc, rb = ctx.solve_batch([ev, ev])
    ctx.set_log(None)
    ctx.solve(ev)                                    # not logged
    lines = [json.loads(l) for l in open(log)]
    assert len(lines) == 3
    assert [l["kind"] for l in lines] == ["single", "batch", "batch"]
    for l, r in zip(lines, [r1] + rb):
        for k in ("D_star", "K_hat", "gap_K", "nodes_expanded", "event_warps", "cell_increments"):
            assert l[k] == r[k], k
        assert l["call_us"] > 0
    ctx.close()


def test_image_at_a_hypothesis_and_pgm(tmp_path):
    w = make_window(64, 48, 32.0, 24.0, 800, 40, 200, 0.3, 0.5, 17)
    ctx = dd.Context(w.W, w.H, w.foe_x, w.foe_y)
    img = ctx.image(dd.Events.of(w, device="cuda"), 0.3)
    want = O.contrast(O.Window.of(w), 0.3, want_iwe=True)[3]
    assert np.array_equal(img, want)
    dd.write_pgm(str(tmp_path / "iwe.pgm"), img)
    assert np.array_equal(dd.read_pgm(str(tmp_path / "iwe.pgm")), img)
    ctx.close()
