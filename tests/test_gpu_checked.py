"""The checked build (-DDD_CHECKED: every tile, event, accumulator and
ingest index tested before use; an index out of range sets a bit of an error
word and the access is skipped) on parity workloads: the results equal the
oracle's and no index is ever out of range.  The stand-in for a memory
checker; run in a child process that loads libdd_checked.so."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA device", allow_module_level=True)

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, sys
import numpy as np
sys.path.insert(0, ROOT)
import oracle as O
import paper_2209_13168_gb300 as dd
from synth import make_window, window_config1, window_config2
from synth.descent import batch_params3, batch_window3
f, checked = dd.dd_check_flags(reset=True)
assert checked and f == 0
def same_images(w, ctx, Ds, lo, hi, **kw):
    win = O.Window.of(w, **kw)
    ev = dd.Events.of(w, device="cuda", polarity=bool(kw.get("polarity")))
    K, S, N, img = ctx.contrast(ev, np.asarray(Ds, np.float32), want_iwe=True)
    for j, D in enumerate(Ds):
        k, s, n, im = O.contrast(win, float(D), want_iwe=True)
        assert (K[j], int(S[j]), int(N[j])) == (k, s, n) and np.array_equal(img[j], im)
    Kb, Sb, Nb, imb = ctx.bound(ev, np.asarray(lo, np.float32), np.asarray(hi, np.float32), want_iwe=True)
    for j in range(len(lo)):
        k, s, n, im = O.bound(win, float(lo[j]), float(hi[j]), want_iwe=True)
        assert (Kb[j], int(Sb[j]), int(Nb[j])) == (k, s, n) and np.array_equal(imb[j], im)
c1, c2 = window_config1(), window_config2()
rag = make_window(97, 61, 48.5, 30.0, 900, 45, 300, 0.45, 0.35, 9)
for w, kw in ((c1, {}), (rag, {"band_rows": 1}), (rag, {"band_rows": 7, "threads": 96})):
    ctx = dd.Context(w.W, w.H, w.foe_x, w.foe_y, **kw)
    same_images(w, ctx, [-1.0, 0.0, 0.2, 0.45, 1.0], [-1.0, 0.1, 0.44], [1.0, 0.3, 0.4501])
    ctx.close()
# wide bounds split over several blocks and merged in the accumulator
ctx = dd.Context(c2.W, c2.H, c2.foe_x, c2.foe_y, max_splits=16)
same_images(c2, ctx, [0.35], [-1.0, 0.0], [1.0, 0.7])
ctx.close()
# polarity planes
ctx = dd.Context(c1.W, c1.H, c1.foe_x, c1.foe_y, polarity=1)
same_images(c1, ctx, [0.0, 0.2], [0.1], [0.3], polarity=True)
ctx.close()
# searches with traces
for w, pk in ((c1, 4), (c2, 16)):
    ctx = dd.Context(w.W, w.H, w.foe_x, w.foe_y, pop_k=pk)
    got = ctx.solve(dd.Events.of(w, device="cuda"), trace_cap=4096)
    want = O.solve(O.Window.of(w), -1.0, 1.0, 1e-4, 0.0, pk, trace_cap=4096)
    for k in ("D_star", "K_hat", "gap_K", "nodes_expanded", "rounds"):
        assert got[k] == want[k], k
    assert got["trace"] == want["trace"]
    ctx.close()
p = batch_params3()
ws = [batch_window3(i, p) for i in (142, 68, 62)]
ctx = dd.Context(640, 480, 320.0, 240.0, pop_k=8)
rc, res = ctx.solve_batch([dd.Events.of(w, device="cuda") for w in ws])
assert rc == dd.DD_OK
for w, r in zip(ws, res):
    assert r["K_hat"] == O.solve(O.Window.of(w), -1.0, 1.0, 1e-4, 0.0, 8)["K_hat"]
ctx.close()
f, checked = dd.dd_check_flags()
print(json.dumps({"flags": f, "checked": checked}))
'''


def test_checked_build_parity_and_no_index_out_of_range():
    sys.path.insert(0, os.path.join(ROOT, "paper_2209_13168_gb300"))
    import _build
    lib = _build.build(checked=True)
    env = dict(os.environ, DD_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", "ROOT = %r\n" % ROOT + CHILD], env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    out = json.loads(r.stdout.strip().splitlines()[-1])
    assert out == {"flags": 0, "checked": True}


def test_normal_build_reports_no_checks():
    import paper_2209_13168_gb300 as dd
    assert dd.dd_check_flags() == (0, False)


def test_checked_build_on_random_configurations():
    # the randomised parity cases (every knob, FOE on the frame's edges,
    # polarity, start-of-window warp; single windows and batches) on the
    # checked build: each compares with the oracle and asserts that no index
    # was out of range
    sys.path.insert(0, os.path.join(ROOT, "paper_2209_13168_gb300"))
    import _build
    env = dict(os.environ, DD_LIBRARY=_build.build(checked=True))
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(ROOT, "tests", "test_gpu_fuzz.py"),
                        os.path.join(ROOT, "tests", "test_gpu_batch_fuzz.py"), "-q", "-x", "-p", "no:cacheprovider"],
                       env=env, cwd=ROOT, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert " passed" in r.stdout and "failed" not in r.stdout and "skipped" not in r.stdout
