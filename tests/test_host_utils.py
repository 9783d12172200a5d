"""Host-side utilities of the binding (no GPU): PGM images of counts and the
autotuned-knob lookup."""
import numpy as np

import paper_2209_13168_gb300 as dd


def test_pgm_roundtrip_and_saturation(tmp_path):
    img = np.arange(12, dtype=np.uint32).reshape(3, 4) * 9000
    p = tmp_path / "iwe.pgm"
    dd.write_pgm(str(p), img)
    back = dd.read_pgm(str(p))
    assert back.shape == (3, 4)
    assert np.array_equal(back, np.minimum(img, 65535))
    assert open(p, "rb").read(2) == b"P5"


def test_autotune_lookup_picks_the_nearest_bucket(tmp_path, monkeypatch):
    # Tuned knobs are keyed by geometry, power-of-two event bucket, mode and
    # GPU; a size between buckets takes the nearest bucket (in log2) of the
    # same geometry, mode and GPU, and nothing else.
    import json
    from paper_2209_13168_gb300 import autotune as at
    monkeypatch.setattr(at, "gpu_name", lambda: "GPU_X")
    knobs = lambda r: {"band_rows": r, "threads": 256, "pop_k": 16, "max_splits": 4}
    table = {at.key(640, 480, 4096, "single", "GPU_X"): knobs(8),
             at.key(640, 480, 131072, "single", "GPU_X"): knobs(16),
             at.key(640, 480, 131072, "batch", "GPU_X"): knobs(24),
             at.key(640, 480, 131072, "single", "GPU_Y"): knobs(38),
             at.key(320, 240, 131072, "single", "GPU_X"): knobs(10)}
    p = tmp_path / "tuned.json"
    p.write_text(json.dumps(table))
    assert at.size_bucket(100_000) == 131072 and at.size_bucket(5000) == 4096 and at.size_bucket(0) == 1
    assert at.lookup(640, 480, 100_000, "single", str(p))["band_rows"] == 16      # its own bucket
    assert at.lookup(640, 480, 3000, "single", str(p))["band_rows"] == 8          # nearest below
    assert at.lookup(640, 480, 2_000_000, "single", str(p))["band_rows"] == 16    # nearest above
    assert at.lookup(640, 480, 100_000, "batch", str(p))["band_rows"] == 24       # mode kept apart
    assert at.lookup(1280, 720, 100_000, "single", str(p)) is None                # no such geometry
    monkeypatch.setattr(at, "gpu_name", lambda: "GPU_Z")
    assert at.lookup(640, 480, 100_000, "single", str(p)) is None                 # another GPU


def test_events_marshalling_rejects_what_it_cannot_pass():
    # The C side reads n entries of every array: lengths must agree, and
    # values the ABI's types cannot hold are an error rather than a cast.
    import pytest
    ok = dd.Events([1, 2], [3, 4], [0.1, 0.2], 0.0, 0.5)
    assert ok.x.dtype == np.int16 and ok.t.dtype == np.float32 and ok.c.n == 2
    assert dd.Events(np.array([1.0, 2.0]), [3, 4], [0.1, 0.2], 0.0, 0.5).x.tolist() == [1, 2]
    assert dd.Events([], [], [], 0.0, 0.5).c.n == 0
    for bad in (([1, 2], [3], [0.1, 0.2]),             # a short array
                ([1, 2], [3, 4], [0.1]),
                ([1.5, 2], [3, 4], [0.1, 0.2]),        # not a pixel coordinate
                ([40000, 2], [3, 4], [0.1, 0.2]),      # beyond int16
                ([[1, 2]], [[3, 4]], [0.1, 0.2])):     # not 1-D
        with pytest.raises(ValueError):
            dd.Events(*bad, 0.0, 0.5)
    with pytest.raises(ValueError):
        dd.Events([1], [2], [0.1], 0.0, 0.5, p=[300])   # beyond int8
    with pytest.raises(ValueError):
        dd.Events([1, 2], [3, 4], [0.1, 0.2], 0.0, 0.5, p=[1])
