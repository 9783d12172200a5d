"""Host-side utilities of the binding (no GPU): PGM images of counts."""
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
