"""Pins of the oracle's reference-time variant: events warped to t_ref (the
paper warps to the window's end, t_ref = tau; t_ref = 0 warps to its start,
where the scale 1 - D t is linear in D).

Checked against closed forms (events at the reference time never move), the
inverse of the generator's motion (known-D recovery), and exhaustive search
(the breakpoint sweep with the same reference time, against BnB)."""
import numpy as np
import pytest

import oracle as O
from synth import make_window, window_config1


def tiny(seed, W=29, H=23, n=150, tau=0.5, foe=(14.0, 11.0), t_ref=0.0, t_mode="uniform"):
    rng = np.random.default_rng(seed)
    x = rng.integers(0, W, n)
    y = rng.integers(0, H, n)
    t = (rng.random(n) * tau).astype(np.float32) if t_mode == "uniform" else np.full(n, t_mode, np.float32)
    return O.Window(W, H, foe[0], foe[1], x, y, t, 0.0, tau, t_ref)


def test_events_at_the_reference_time_do_not_move(oracle_lib):
    # t_ref = 0 and every t = 0: s = 1 for every D, so the image is the raw
    # event histogram, the contrast is constant, and the root bound equals it:
    # Algorithm 1 stops without expanding (the mirror of all t = tau for the
    # paper's warp).
    win = tiny(3, t_mode=0.0)
    ks = {O.contrast(win, D)[0] for D in (-1.0, -0.3, 0.0, 0.4, 1.0)}
    assert len(ks) == 1
    r = O.solve(win, -1.0, 1.0, 1e-4, 0.0, 1)
    assert r["nodes_expanded"] == 0 and r["K_hat"] == ks.pop()


def test_linear_warp_cells(oracle_lib):
    # At t_ref = 0 an event moves to FOE + d (1 - D t): one binary32 product,
    # one difference, one product (g = 1 exactly).
    win = tiny(5)
    for D in (-0.7, 0.3, 1.2):
        ux, uy = O.warp_cells(win, D)
        s = (np.float32(1) - np.float32(D) * win.t).astype(np.float32)
        dx = (win.x.astype(np.float32) - np.float32(14.0)).astype(np.float32)
        want = np.floor((np.float32(14.0) + (dx * s).astype(np.float32)).astype(np.float32) + np.float32(0.5))
        assert np.array_equal(ux, want.astype(np.int32))


@pytest.mark.parametrize("K_pop", [1, 4])
def test_bnb_agrees_with_the_sweep_at_t_ref_0(oracle_lib, K_pop):
    rng = np.random.default_rng(60 + K_pop)
    for seed in range(5):
        W, H = int(rng.integers(10, 33)), int(rng.integers(10, 33))
        win = tiny(400 + seed, W=W, H=H, n=int(rng.integers(20, 200)), foe=(float(W // 2), float(H // 2)))
        Kmax, _, _ = O.sweep_max(win, -1.0, 1.0)
        assert O.grid_max(win, -1.0, 1.0, 2.5e-5)[0] <= Kmax
        r = O.solve(win, -1.0, 1.0, 1e-4, 0.0, K_pop)
        assert O.contrast(win, r["D_star"])[0] == r["K_hat"]
        assert r["K_hat"] <= Kmax <= r["K_hat"] + r["gap_K"]


def test_recovers_known_D_at_t_ref_0(oracle_lib):
    # Warping to the start inverts the generator's motion x = FOE + (x0 - FOE)/(1 - D t):
    # at the true D every event of a scene point lands on x0.
    w = make_window(346, 260, 173.0, 130.0, 3000, 150, 0, 0.2, 0.5, 1000)
    r = O.solve(O.Window.of(w, t_ref=0.0), -1.0, 1.0, 1e-4, 0.0, 8)
    assert abs(r["D_star"] - 0.2) <= 0.005
    wn = window_config1()
    r = O.solve(O.Window.of(wn, t_ref=0.0), -1.0, 1.0, 1e-4, 0.0, 8)
    assert abs(r["D_star"] - 0.2) <= 0.02


def test_intermediate_reference_time_and_bad_values(oracle_lib):
    # Any t_ref in [0, tau] is a valid warp target; outside it is refused.
    win = tiny(7, t_ref=0.25)
    Kmax, _, _ = O.sweep_max(win, -1.0, 1.0)
    r = O.solve(win, -1.0, 1.0, 1e-4, 0.0, 2)
    assert r["K_hat"] <= Kmax <= r["K_hat"] + r["gap_K"]
    for bad in (-0.1, 0.6):
        with pytest.raises(O.OracleError):
            O.contrast(tiny(8, t_ref=bad), 0.1)
