"""Pins of the oracle's per-polarity objective: one image per polarity and the
sum of their contrasts (the paper leaves polarity out of Eq. 12 and notes it
could be used).

Checked against the paper's single-image objective, which it must reduce to
when every event has one polarity, and which it must equal plane by plane on
the window split by polarity (the two planes are two independent windows
whose keys add); against exhaustive search (the breakpoint sweep over the same
objective, against BnB); and against the generator's known D."""
import numpy as np
import pytest

import oracle as O
from synth import window_config1


def tiny(seed, W=29, H=23, n=150, tau=0.5, foe=(14.0, 11.0), p_mode="random"):
    rng = np.random.default_rng(seed)
    x = rng.integers(0, W, n)
    y = rng.integers(0, H, n)
    t = (rng.random(n) * tau).astype(np.float32)
    p = {"random": rng.choice(np.array([-1, 1], np.int8), n), "on": np.ones(n, np.int8),
         "off": -np.ones(n, np.int8)}[p_mode]
    return x, y, t, p, dict(W=W, H=H, foe_x=foe[0], foe_y=foe[1], t0=0.0, tau=tau)


def win(x, y, t, g, p=None, t_ref=None):
    return O.Window(g["W"], g["H"], g["foe_x"], g["foe_y"], x, y, t, g["t0"], g["tau"], t_ref, p)


@pytest.mark.parametrize("p_mode,plane", [("on", 0), ("off", 1)])
def test_one_polarity_is_the_paper_objective(oracle_lib, p_mode, plane):
    x, y, t, p, g = tiny(2, p_mode=p_mode)
    a, b = win(x, y, t, g), win(x, y, t, g, p)
    for D in (-0.8, 0.0, 0.3, 1.1):
        k, s, n, im = O.contrast(a, D, want_iwe=True)
        kp, sp, np_, imp = O.contrast(b, D, want_iwe=True)
        assert (k, s, n) == (kp, sp, np_)
        assert np.array_equal(imp[plane], im) and not imp[1 - plane].any()
    for lo, hi in ((-1.0, 1.0), (0.2, 0.3), (0.5, 0.50001)):
        assert O.bound(a, lo, hi)[:3] == O.bound(b, lo, hi)[:3]
    ra = O.solve(a, -1.0, 1.0, 1e-4, 0.0, 2, trace_cap=512)
    rb = O.solve(b, -1.0, 1.0, 1e-4, 0.0, 2, trace_cap=512)
    assert ra == rb


@pytest.mark.parametrize("t_ref", [None, 0.0])
def test_planes_are_two_windows_whose_keys_add(oracle_lib, t_ref):
    for seed in range(4):
        x, y, t, p, g = tiny(10 + seed, n=200 + 40 * seed)
        on, off = p > 0, p <= 0
        both = win(x, y, t, g, p, t_ref)
        a, b = win(x[on], y[on], t[on], g, None, t_ref), win(x[off], y[off], t[off], g, None, t_ref)
        for D in (-0.6, 0.1, 0.45, 0.9):
            k, s, n, im = O.contrast(both, D, want_iwe=True)
            ka, sa, na, ima = O.contrast(a, D, want_iwe=True)
            kb, sb, nb, imb = O.contrast(b, D, want_iwe=True)
            assert (k, s, n) == (ka + kb, sa + sb, na + nb)
            assert np.array_equal(im[0], ima) and np.array_equal(im[1], imb)
        for lo, hi in ((-1.0, 1.0), (0.05, 0.4), (0.3, 0.3005)):
            k, s, n, im = O.bound(both, lo, hi, want_iwe=True)
            ka, sa, na, ima = O.bound(a, lo, hi, want_iwe=True)
            kb, sb, nb, imb = O.bound(b, lo, hi, want_iwe=True)
            assert (k, s, n) == (ka + kb, sa + sb, na + nb)
            assert np.array_equal(im[0], ima) and np.array_equal(im[1], imb)


def test_polarity_encodings_and_flip(oracle_lib):
    # {0, 1} and {-1, +1} encode the same split (p <= 0 is the second plane);
    # flipping every polarity swaps the planes and keeps the key.
    x, y, t, p, g = tiny(31)
    a = win(x, y, t, g, p)
    b = win(x, y, t, g, (p > 0).astype(np.int8))
    c = win(x, y, t, g, -p)
    for D in (-0.3, 0.25):
        ka, _, _, ia = O.contrast(a, D, want_iwe=True)
        kb, _, _, ib = O.contrast(b, D, want_iwe=True)
        kc, _, _, ic = O.contrast(c, D, want_iwe=True)
        assert ka == kb == kc
        assert np.array_equal(ia, ib) and np.array_equal(ia[::-1], ic)


def test_bound_dominates_the_contrast(oracle_lib):
    rng = np.random.default_rng(5)
    x, y, t, p, g = tiny(41, n=300)
    w = win(x, y, t, g, p)
    for _ in range(10):
        lo = float(rng.uniform(-1.0, 0.9))
        hi = float(min(1.0, lo + 10 ** rng.uniform(-4, 0)))
        kb = O.bound(w, lo, hi)[0]
        for D in np.linspace(lo, hi, 17, dtype=np.float32):
            assert O.contrast(w, float(D))[0] <= kb


@pytest.mark.parametrize("K_pop", [1, 4])
def test_bnb_agrees_with_the_sweep_with_polarity(oracle_lib, K_pop):
    rng = np.random.default_rng(80 + K_pop)
    for seed in range(5):
        W, H = int(rng.integers(10, 33)), int(rng.integers(10, 33))
        x, y, t, p, g = tiny(500 + seed, W=W, H=H, n=int(rng.integers(20, 200)), foe=(float(W // 2), float(H // 2)))
        w = win(x, y, t, g, p)
        Kmax, _, _ = O.sweep_max(w, -1.0, 1.0)
        r = O.solve(w, -1.0, 1.0, 1e-4, 0.0, K_pop)
        assert O.contrast(w, r["D_star"])[0] == r["K_hat"]
        assert r["K_hat"] <= Kmax <= r["K_hat"] + r["gap_K"]


def test_recovers_known_D_with_polarity(oracle_lib):
    w = window_config1()
    r = O.solve(O.Window.of(w, polarity=True), -1.0, 1.0, 1e-4, 0.0, 8)
    assert abs(r["D_star"] - 0.2) <= 0.02
