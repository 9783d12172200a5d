"""Pins of the CPU oracle against facts the paper and the mathematics fix.

Nothing here compares the oracle with itself: each test checks it against a
closed form, a library routine applied to an independently built image, a
hand-derived case, or exhaustive search (McLeod et al., arXiv 2209.13168).
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
from synth import make_window, window_config1

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def tiny(seed, W=29, H=23, n=120, tau=0.5, foe=(14.0, 11.0), t_mode="uniform"):
    rng = np.random.default_rng(seed)
    x = rng.integers(0, W, n).astype(np.int16)
    y = rng.integers(0, H, n).astype(np.int16)
    if t_mode == "uniform":
        t = (rng.random(n) * tau).astype(np.float32)
    elif t_mode == "zero":
        t = np.zeros(n, np.float32)
    else:
        t = np.full(n, tau, np.float32)
    return O.Window(W, H, foe[0], foe[1], x, y, t, 0.0, tau)


def hist(win, ux, uy):
    img = np.zeros((win.H, win.W), np.int64)
    ok = (ux >= 0) & (ux < win.W) & (uy >= 0) & (uy < win.H)
    np.add.at(img, (uy[ok], ux[ok]), 1)
    return img


# ------------------------------------------------------------ closed forms

def test_single_event_key(oracle_lib):
    # Eq. (13) with one in-frame event: mean 1/M, C = 1/M - 1/M^2, so M^2 C = M - 1.
    win = O.Window(40, 30, 20.0, 15.0, [23], [13], [0.1], 0.0, 0.5)
    for D in (-0.7, 0.0, 0.3, 1.2):
        K, S, N, _ = O.contrast(win, D)
        assert (K, S, N) == (win.M - 1, 1, 1)


def test_events_on_foe_one_pixel(oracle_lib):
    # Events on the FOE never move: all n in one pixel, M^2 C = M n^2 - n^2, for
    # every D; the bound image has the same single pixel on every interval.
    n = 17
    t = np.linspace(0, 0.4, n).astype(np.float32)
    win = O.Window(33, 21, 16.0, 10.0, [16] * n, [10] * n, t, 0.0, 0.4)
    want = win.M * n * n - n * n
    for D in (-1.0, 0.25, 1.5):
        assert O.contrast(win, D)[0] == want
    for lo, hi in ((-1.0, 1.0), (0.1, 0.11), (1.0, 1.8)):
        Kb, Sb, Nf, img = O.bound(win, lo, hi, want_iwe=True)
        assert (Kb, Sb, Nf) == (want, n * n, n)
        assert img.sum() == n and img[10, 16] == n


def test_contrast_is_population_variance(oracle_lib):
    # Eq. (13): C is the variance of H over all M pixels (mean over all M).
    # Build H independently from the warped cells and use numpy's variance.
    for seed in range(5):
        win = tiny(seed, W=31, H=19, n=300)
        for D in (-0.9, 0.0, 0.37, 1.1):
            K, S, N, img = O.contrast(win, D, want_iwe=True)
            ux, uy = O.warp_cells(win, D)
            H = hist(win, ux, uy)
            assert np.array_equal(img, H)
            C = np.var(H.astype(np.float64))
            assert math.isclose(K, C * win.M ** 2, rel_tol=1e-12, abs_tol=1e-6)
            assert N == H.sum() and S == (H * H).sum()


def test_identity_warp_at_D0(oracle_lib):
    # D = 0 gives s = 1: every event stays in its own pixel (Eq. (11)).
    for seed in range(4):
        win = tiny(seed, n=200)
        ux, uy = O.warp_cells(win, 0.0)
        assert np.array_equal(ux, win.x) and np.array_equal(uy, win.y)
        img = O.contrast(win, 0.0, want_iwe=True)[3]
        assert np.array_equal(img, hist(win, win.x.astype(np.int64), win.y.astype(np.int64)))


def test_time_origin_is_the_window_start(oracle_lib):
    # Sec. 3.3: a batch's times count from its start, so moving every t and
    # t0 by the same amount changes nothing.  Times on a 2^-12 grid and
    # t0 = 2 keep every t - t0 exact in binary32.
    rng = np.random.default_rng(12)
    W, H, n, tau = 33, 27, 250, 0.5
    x = rng.integers(0, W, n).astype(np.int16)
    y = rng.integers(0, H, n).astype(np.int16)
    t = (rng.integers(0, 2048, n) / 4096.0).astype(np.float32)
    a = O.Window(W, H, 16.0, 13.0, x, y, t, 0.0, tau)
    b = O.Window(W, H, 16.0, 13.0, x, y, (t + np.float32(2.0)).astype(np.float32), 2.0, tau)
    assert np.array_equal((b.t - np.float32(2.0)).astype(np.float32), t)
    for D in (-0.8, 0.3, 1.2):
        assert O.contrast(a, D)[:3] == O.contrast(b, D)[:3]
        assert np.array_equal(O.warp_cells(a, D)[0], O.warp_cells(b, D)[0])
    for lo, hi in ((-1.0, 1.0), (0.2, 0.3)):
        assert O.bound(a, lo, hi)[:3] == O.bound(b, lo, hi)[:3]
    ra, rb = O.solve(a, -1.0, 1.0, 1e-4, 0.0, 2), O.solve(b, -1.0, 1.0, 1e-4, 0.0, 2)
    assert (ra["D_star"], ra["K_hat"], ra["nodes_expanded"]) == (rb["D_star"], rb["K_hat"], rb["nodes_expanded"])


@pytest.mark.parametrize("D,g", [(1.0, 2), (1.5, 4)])
def test_zoom_when_all_t_zero(oracle_lib, D, g):
    # t_i = 0 makes the warp a pure zoom about the FOE by g = 1/(1 - D tau);
    # tau = 0.5 and D in {1, 1.5} give g in {2, 4}, exact in binary32.  A
    # half-integer FOE puts zoomed points on pixel borders: x' = g x - (g-1) foe,
    # and a point on a border belongs to the pixel above it ([u-1/2, u+1/2)).
    W, H = 37, 26  # W != H catches swapped axes
    rng = np.random.default_rng(7)
    x = rng.integers(0, W, 150)
    y = rng.integers(0, H, 150)
    fx, fy = 18.5, 12.0
    win = O.Window(W, H, fx, fy, x, y, np.zeros(150, np.float32), 0.0, 0.5)
    ux, uy = O.warp_cells(win, D)
    ex = np.floor(g * x - (g - 1) * fx + 0.5).astype(np.int64)
    ey = np.floor(g * y - (g - 1) * fy + 0.5).astype(np.int64)
    assert np.array_equal(ux, ex) and np.array_equal(uy, ey)
    # explicit half-pixel case: x = 19, foe 18.5, g = 2 -> 19.5 -> pixel 20
    one = O.Window(W, H, fx, fy, [19], [12], [0.0], 0.0, 0.5)
    assert O.warp_cells(one, 1.0)[0][0] == 20


def test_all_t_tau_is_constant(oracle_lib):
    # t_i = tau gives s = 1 for every D: C is constant, the bound is exact on
    # any interval (the segment is a point), and Algorithm 1 stops at once.
    win = tiny(3, n=250, t_mode="tau")
    K0 = O.contrast(win, 0.0)[0]
    for D in (-1.0, 0.2, 1.4):
        assert O.contrast(win, D)[0] == K0
    for lo, hi in ((-1.0, 1.5), (0.3, 0.31)):
        assert O.bound(win, lo, hi)[0] == K0
    r = O.solve(win, -1.0, 1.5, 1e-4, 0.0, 1)
    assert r["nodes_expanded"] == 0 and r["K_hat"] == K0 and r["gap_K"] == 0


def test_two_event_plateau_golden(oracle_lib):
    # Hand-derived worked case (Eq. (11)): golden/two_event_plateau.json.
    g = json.load(open(os.path.join(GOLDEN, "two_event_plateau.json")))
    win = O.Window(g["W"], g["H"], g["foe"][0], g["foe"][1], g["x"], g["y"], g["t"], 0.0, g["tau"])
    M = win.M
    lo, hi = g["plateau"]
    for D in np.linspace(-1.0, 1.45, 491):
        D = float(np.float32(D))
        if abs(D - lo) < 1e-5 or abs(D - hi) < 1e-5:
            continue
        K = O.contrast(win, D)[0]
        assert K == (4 * M - 4 if lo <= D < hi else 2 * M - 4), D
    r = O.solve(win, -1.0, 1.45, 1e-4, 0.0, 1)
    assert r["K_hat"] == 4 * M - 4 and lo <= r["D_star"] < hi
    assert lo <= g["D_coincide"] < hi


# ------------------------------------------------------------- invariants

def _samples(lo, hi, rng):
    lo32, hi32 = np.float32(lo), np.float32(hi)
    pts = [lo32, hi32, np.nextafter(lo32, np.float32(np.inf)), np.nextafter(hi32, np.float32(-np.inf)),
           np.float32(lo32 + np.float32(0.5) * (hi32 - lo32))]
    pts += list((lo + rng.random(59) * (hi - lo)).astype(np.float32))
    return [float(np.clip(p, lo32, hi32)) for p in pts]


def test_bound_dominates_contrast(oracle_lib):
    # Eqs. (15)-(19): Hbar >= H pixelwise, N_full <= N_in(D), Kbar >= K(D),
    # for 64 binary32 D per interval (ends, their inner neighbours, centre).
    rng = np.random.default_rng(11)
    for seed in range(12):
        win = tiny(100 + seed, W=int(rng.integers(8, 40)), H=int(rng.integers(8, 40)),
                   n=int(rng.integers(1, 150)), tau=float(rng.uniform(0.1, 0.6)),
                   foe=(float(rng.integers(0, 8)) + 0.5 * int(rng.integers(0, 2)), 4.0))
        for _ in range(6):
            a, b = sorted(rng.uniform(-1.0, 0.75 / win.c.tau, 2))
            if rng.random() < 0.5:
                b = a + 10 ** rng.uniform(-6, -2)
            a, b = float(np.float32(a)), float(np.float32(min(b, 0.75 / win.c.tau)))
            if not a < b:
                continue
            Kb, Sb, Nf, Hb = O.bound(win, a, b, want_iwe=True)
            for D in _samples(a, b, rng):
                K, S, N, Hp = O.contrast(win, D, want_iwe=True)
                assert K <= Kb and S <= Sb and Nf <= N
                assert (Hb >= Hp).all()
                assert Hp.sum() == N


def test_scale_interval_contains_every_binary32_scale(oracle_lib):
    # The real s(D) is monotone in D (ds/dD = (tau - t)/(1 - D tau)^2 >= 0) but
    # its binary32 value is not, at the ulp level.  The widened interval must
    # still contain s(D) for every binary32 D in [D_lo, D_hi]; check the 300
    # binary32 values next to each end and 200 interior ones.
    rng = np.random.default_rng(17)
    f = np.float32
    for trial in range(400):
        tau = float(f(rng.uniform(0.05, 0.6)))
        t = float(f(f(rng.random()) * f(tau)))
        if trial % 10 == 0:
            t = tau if trial % 20 == 0 else 0.0
        a, b = sorted(rng.uniform(-64.0 / tau if trial % 7 == 0 else -1.5, 0.75 / tau, 2))
        if trial % 3 == 0:
            b = a + 10 ** rng.uniform(-7, -3)
        a, b = f(a), f(min(b, 0.75 / tau))
        if not a < b:
            continue
        sa, sb = O.scale_interval(float(a), float(b), t, tau)
        Ds = [a, b]
        lo, hi = a, b
        for _ in range(300):
            lo, hi = np.nextafter(lo, f(np.inf)), np.nextafter(hi, f(-np.inf))
            Ds += [lo, hi]
        Ds += list(f(a + rng.random(200) * (float(b) - float(a))))
        for D in Ds:
            if a <= D <= b:
                assert sa <= O.scale(float(D), t, tau) <= sb, (trial, float(D))


def _seg_cell_dist(p0, p1, k, j):
    # distance from segment p0-p1 to the closed pixel square [k-1/2,k+1/2]x[j-1/2,j+1/2]
    ts = np.linspace(0.0, 1.0, 4001)
    px = p0[0] + (p1[0] - p0[0]) * ts
    py = p0[1] + (p1[1] - p0[1]) * ts
    dx = np.maximum(np.abs(px - k) - 0.5, 0.0)
    dy = np.maximum(np.abs(py - j) - 0.5, 0.0)
    return float(np.sqrt(dx * dx + dy * dy).min())


def test_bound_rasterisation_matches_real_segment(oracle_lib):
    # Eq. (16) for single events: every pixel the real segment
    # f(D_lo) <-> f(D_hi) passes through is covered, and every covered pixel
    # lies within the 2^-8 px margin (plus the 2^-19 scale widening) of it.
    rng = np.random.default_rng(5)
    W, H, fx, fy, tau = 48, 40, 24.0, 20.0, 0.5
    for trial in range(150):
        x, y = int(rng.integers(0, W)), int(rng.integers(0, H))
        t = float(np.float32(rng.uniform(0, tau)))
        a, b = sorted(rng.uniform(-1.0, 1.5, 2))
        a, b = float(np.float32(a)), float(np.float32(b))
        if not a < b:
            continue
        win = O.Window(W, H, fx, fy, [x], [y], [t], 0.0, tau)
        Kb, Sb, Nf, Hb = O.bound(win, a, b, want_iwe=True)
        s = lambda D: (1 - D * t) / (1 - D * tau)
        p0 = (fx + (x - fx) * s(a), fy + (y - fy) * s(a))
        p1 = (fx + (x - fx) * s(b), fy + (y - fy) * s(b))
        # Eqs. (18)-(19) for one event: each covered pixel holds 1, so
        # Sbar = L (the covered count), and N_full is 1 exactly when the
        # whole segment lies in the frame (decided here in binary64, away
        # from the frame's edges).
        L = int(Hb.sum())
        inside = [-0.5 + 1e-3 <= p[0] <= W - 0.5 - 1e-3 and -0.5 + 1e-3 <= p[1] <= H - 0.5 - 1e-3 for p in (p0, p1)]
        outside = [not (-0.5 - 1e-3 <= p[0] <= W - 0.5 + 1e-3 and -0.5 - 1e-3 <= p[1] <= H - 0.5 + 1e-3)
                   for p in (p0, p1)]
        if all(inside):
            assert Nf == 1, trial
        if any(outside):
            assert Nf == 0, trial
        assert Sb == L and Kb == win.M * L - Nf, trial
        ts = np.linspace(0.0, 1.0, 20001)
        cx = np.floor(p0[0] + (p1[0] - p0[0]) * ts + 0.5).astype(int)
        cy = np.floor(p0[1] + (p1[1] - p0[1]) * ts + 0.5).astype(int)
        ok = (cx >= 0) & (cx < W) & (cy >= 0) & (cy < H)
        assert (Hb[cy[ok], cx[ok]] == 1).all(), trial
        assert Hb.max() <= 1
        for j, k in zip(*np.nonzero(Hb)):
            assert _seg_cell_dist(p0, p1, k, j) <= 2 ** -8 + 1e-3, (trial, k, j)


def test_leaf_free_bound_shrinks_to_point(oracle_lib):
    # Equality in the limit (Eq. (17) and the proof of Eq. (19)): on a tiny
    # interval that straddles no pixel border, Kbar = K(D).
    win = tiny(9, n=80)
    hits = 0
    for D in np.linspace(-0.8, 1.3, 40):
        D = float(np.float32(D))
        Kb = O.bound(win, D, float(np.nextafter(np.float32(D), np.float32(2))))[0]
        if Kb == O.contrast(win, D)[0]:
            hits += 1
    assert hits >= 35


# ------------------------------------------------------------ brute force

def test_sweep_is_exhaustive_on_a_narrow_interval(oracle_lib):
    # Every binary32 D in [lo, hi] enumerated one by one.
    win = tiny(21, W=24, H=20, n=60, foe=(12.0, 10.0))
    lo = np.float32(0.3)
    D = [lo]
    while len(D) < 6000:
        D.append(np.nextafter(D[-1], np.float32(1)))
    hi = float(D[-1])
    best = max(O.contrast(win, float(d))[0] for d in D)
    assert O.sweep_max(win, float(lo), hi)[0] == best
    win2 = tiny(22, W=24, H=20, n=60, foe=(12.0, 10.0))
    lo = np.float32(-0.21)
    D = [lo]
    while len(D) < 6000:
        D.append(np.nextafter(D[-1], np.float32(1)))
    best = max(O.contrast(win2, float(d))[0] for d in D)
    assert O.sweep_max(win2, float(lo), float(D[-1]))[0] == best


def test_sweep_finds_a_sliver_next_to_a_breakpoint(oracle_lib):
    # Two events in one pixel column whose warps share a pixel on only 4
    # binary32 values of D, next to a real breakpoint: the binary32 warp
    # changes pixel a few ulps away from the real crossing, so a sweep that
    # only looked at breakpoints and the midpoints between them would miss
    # the maximum.  Every binary32 D of the interval enumerated one by one.
    win = O.Window(40, 8, 4.0, 4.0, [35, 35], [4, 4], [0.435791015625, 0.307373046875], 0.0, 0.5)
    lo, hi = np.float32(-0.2872776687145233), np.float32(-0.287276953458786)
    D = [lo]
    while D[-1] < hi:
        D.append(np.nextafter(D[-1], np.float32(1)))
    K = [O.contrast(win, float(d))[0] for d in D]
    best = max(K)
    assert best == 4 * win.M - 4 and K.count(best) <= 4
    assert O.sweep_max(win, float(lo), float(hi))[0] == best


def test_grid_is_its_definition(oracle_lib):
    # The dense grid: the contrast at D_lo + j h (binary64, rounded to
    # binary32) for j = 0, 1, ... while it stays within [D_lo, D_hi], plus
    # D_hi itself; the largest key and the smallest D attaining it.
    # The two-event plateau of golden/two_event_plateau.json, [6/11, 10/13),
    # is first reached at an odd grid point from 0.45 in steps of 0.1.
    g = json.load(open(os.path.join(GOLDEN, "two_event_plateau.json")))
    plateau = O.Window(g["W"], g["H"], g["foe"][0], g["foe"][1], g["x"], g["y"], g["t"], 0.0, g["tau"])
    for win, lo, hi, h in ((tiny(31, W=27, H=21, n=90), -0.75, 0.5, 0.0625), (plateau, 0.45, 0.9, 0.1)):
        steps = int(math.floor((np.float64(np.float32(hi)) - np.float64(np.float32(lo))) /
                               np.float64(np.float32(h))))
        Ds = [float(np.float32(np.float64(np.float32(lo)) + j * np.float64(np.float32(h)))) for j in range(steps + 1)]
        Ds.append(float(np.float32(hi)))
        Ks = [O.contrast(win, D)[0] for D in Ds]
        best = max(Ks)
        K, D_at, n = O.grid_max(win, lo, hi, h)
        assert (K, D_at, n) == (best, min(D for D, k in zip(Ds, Ks) if k == best), len(Ds))
    assert K == 4 * plateau.M - 4 and abs(D_at - 0.55) < 1e-6


def test_grid_includes_its_upper_end(oracle_lib):
    # The dense grid evaluates D_lo + j h and D_hi itself: on an interval
    # that enters the two-event plateau of golden/two_event_plateau.json by
    # less than one step, only the upper end finds the plateau's K.
    g = json.load(open(os.path.join(GOLDEN, "two_event_plateau.json")))
    win = O.Window(g["W"], g["H"], g["foe"][0], g["foe"][1], g["x"], g["y"], g["t"], 0.0, g["tau"])
    hi = float(np.float32(g["plateau"][0] + 0.001))
    lo = float(np.float32(hi - 0.0195))
    K, D_at, n = O.grid_max(win, lo, hi, 0.01)
    assert (K, D_at, n) == (4 * win.M - 4, hi, 3)


@pytest.mark.parametrize("K_pop", [1, 3, 8])
def test_bnb_agrees_with_brute_force(oracle_lib, K_pop):
    # Algorithm 1 returns a K it attained, and its certificate covers the
    # exhaustive maximum: K_hat <= K_max <= K_hat + gap_K.
    rng = np.random.default_rng(31 + K_pop)
    for seed in range(6):
        W, H = int(rng.integers(10, 33)), int(rng.integers(10, 33))
        win = tiny(200 + seed, W=W, H=H, n=int(rng.integers(20, 200)), tau=0.5,
                   foe=(float(W // 2), float(H // 2)))
        lo, hi = -1.0, 1.0
        r = O.solve(win, lo, hi, 1e-4, 0.0, K_pop)
        Kmax, Dmax, _ = O.sweep_max(win, lo, hi)
        Kgrid, _, _ = O.grid_max(win, lo, hi, 2.5e-5)
        assert O.contrast(win, r["D_star"])[0] == r["K_hat"]
        assert r["K_hat"] <= Kmax <= r["K_hat"] + r["gap_K"]
        assert Kgrid <= Kmax
        assert r["gap_K"] >= 0 and r["bound_gap"] >= 0
        # the reported contrast is Eq. (13) at D*: the variance of its image
        ux, uy = O.warp_cells(win, r["D_star"])
        C = np.var(hist(win, ux, uy).astype(np.float64))
        assert math.isclose(r["contrast"], C, rel_tol=1e-12, abs_tol=1e-15)


@pytest.mark.parametrize("K_pop", [1, 4])
def test_search_counters_rebuilt_from_the_trace(oracle_lib, K_pop):
    # The search's work counters, recounted from its trace: the root's centre
    # and bound, then per expanded interval its centre and, unless it is a
    # leaf, its two halves' bounds, each re-evaluated on its own; the cells
    # are the in-frame events of each centre's image (Eq. 12) and the
    # covered cells of each bound's image (Eq. 16).
    win = tiny(77, W=31, H=23, n=150)
    lo, hi = -1.0, 1.0
    r = O.solve(win, lo, hi, 1e-4, 0.0, K_pop, trace_cap=100000)
    tr = r["trace"]
    assert len(tr) == r["trace_len"] == r["nodes_expanded"]
    c0 = float(np.float32(np.float32(lo) + np.float32(0.5) * (np.float32(hi) - np.float32(lo))))
    points, bounds = [c0] + [t[2] for t in tr], [(lo, hi)]
    for D_lo, D_hi, D_c, leaf, _, _ in tr:
        if not leaf:
            bounds += [(D_lo, D_c), (D_c, D_hi)]
    assert (r["point_evals"], r["bound_evals"]) == (len(points), len(bounds))
    assert r["event_warps"] == win.x.size * (len(points) + len(bounds))
    pc = sum(int(O.contrast(win, D)[2]) for D in points)
    bc = sum(int(O.bound(win, a, b, want_iwe=True)[3].sum()) for a, b in bounds)
    assert (r["cell_increments"], r["bound_increments"]) == (pc + bc, bc)
    if K_pop == 1:
        assert r["rounds"] == r["nodes_expanded"]


@pytest.mark.parametrize("K_pop", [1, 4])
def test_ties_follow_algorithm_1(oracle_lib, K_pop):
    # One event 2 px right of the FOE at t = tau/2 stays in the frame for
    # every D in [-1, 1] (its offset scales by 5/6 to 3/2), so C(D) is the
    # same everywhere (K = M - 1) and every expanded centre ties the
    # incumbent: with Algorithm 1's ">=" each replaces it, and D* is the
    # last centre expanded.  Every child bound is at least M - 1 (the event
    # covers a pixel and the segment stays in the frame), so the ">=" of the
    # insertion queues every child: expanding the root queues both halves,
    # [-1, 0] only tying the incumbent (its segment stays in pixel 18).
    win = O.Window(32, 32, 16.0, 16.0, [18], [16], [0.25], 0.0, 0.5)
    M = win.M
    for D in (-1.0, -0.3, 0.0, 0.6, 1.0):
        assert O.contrast(win, D)[0] == M - 1
    assert O.bound(win, -1.0, 0.0)[0] == M - 1 and O.bound(win, 0.0, 1.0)[0] == 2 * M - 1
    r = O.solve(win, -1.0, 1.0, 1e-4, 0.0, K_pop, trace_cap=4096)
    assert r["nodes_expanded"] > 1 and r["K_hat"] == M - 1
    assert r["D_star"] == r["trace"][-1][2] != 0.0
    assert r["max_queue"] >= 2


def test_pop_k_keeps_the_optimum(oracle_lib):
    # Different pop widths explore differently but certify the same maximum.
    w = window_config1()
    win = O.Window.of(w)
    rs = [O.solve(win, -1.0, 1.0, 1e-4, 0.0, k) for k in (1, 4, 16)]
    for r in rs:
        assert O.contrast(win, r["D_star"])[0] == r["K_hat"]
    lo = max(r["K_hat"] for r in rs)
    assert all(r["K_hat"] + r["gap_K"] >= lo for r in rs)


def test_gamma_stops_early(oracle_lib):
    # The stopping test of Algorithm 1 with gamma > 0: the search stops once the best
    # bound is within gamma (contrast units) of the incumbent.
    win = O.Window.of(window_config1())
    r0 = O.solve(win, -1.0, 1.0, 1e-4, 0.0, 1)
    r1 = O.solve(win, -1.0, 1.0, 1e-4, 0.025, 1)
    assert r1["nodes_expanded"] < r0["nodes_expanded"]
    assert r1["bound_gap"] <= 0.025 + 1e-12
    assert r1["K_hat"] <= r0["K_hat"] + r0["gap_K"]


# ------------------------------------------------------------- recovery

def test_recovers_known_D_noise_free(oracle_lib):
    # The generator's motion is the inverse of the warp, so its D is the
    # noise-free optimum up to the rounding of generated pixel positions.
    for seed, D, tau in ((1, 0.2, 0.5), (2, 0.55, 0.4), (3, -0.3, 0.5)):
        w = make_window(346, 260, 173.0, 130.0, 3000, 150, 0, D, tau, seed)
        r = O.solve(O.Window.of(w), -1.0, 1.0, 1e-4, 0.0, 4)
        assert abs(r["D_star"] - D) <= 0.005, (D, r["D_star"])


def test_recovers_known_D_with_noise(oracle_lib):
    # Tolerance 0.02 s^-1 with 25% noise: an acceptance bound of this build,
    # not a number from the paper.
    w = window_config1()
    r = O.solve(O.Window.of(w), -1.0, 1.0, 1e-4, 0.0, 1)
    assert abs(r["D_star"] - 0.2) <= 0.02


def test_divergence_retrieval(oracle_lib):
    # Sec. 4.1: D* = nu*/(1 + nu* tau); here nu = -D, so D_end = D/(1 - D tau)
    # (sign flipped: positive while approaching).
    win = O.Window.of(window_config1())
    r = O.solve(win, -1.0, 1.0, 1e-4, 0.0, 4)
    nu = -float(r["D_star"])
    paper = nu / (1.0 + nu * 0.5)
    assert math.isclose(r["D_end"], -paper, rel_tol=1e-6)


def _fp64_recount(win, D):
    # the same warp in binary64 with numpy (times relative to t0 as binary32
    # differences, the FOE and D as their binary32 values), against the
    # oracle's binary32 cells
    c = win.c
    ux, uy = O.warp_cells(win, D)
    D64 = float(np.float32(D))
    ti = (win.t - np.float32(c.t0)).astype(np.float32).astype(np.float64)
    sd = (1.0 - D64 * ti) / (1.0 - D64 * float(c.t_ref))
    fx, fy = float(c.foe_x), float(c.foe_y)
    ux64 = np.floor(fx + (win.x.astype(np.float64) - fx) * sd + 0.5).astype(np.int64)
    uy64 = np.floor(fy + (win.y.astype(np.float64) - fy) * sd + 0.5).astype(np.int64)
    return int(((ux64 != ux) | (uy64 != uy)).sum())


@pytest.mark.parametrize("t_ref", [None, 0.0])
def test_fp64_disagreements(oracle_lib, t_ref):
    # The diagnostic counts the events whose binary64 warp lands in another
    # pixel than the binary32 warp: a numpy recount agrees at every D of a
    # sweep, the count is nonzero somewhere (events near pixel borders), and
    # it stays rare (a few events of 4,000).
    win = O.Window.of(window_config1(), t_ref=t_ref)
    counts = []
    for D in np.linspace(-1.0, 1.0, 201):
        n = O.fp64_disagreements(win, float(np.float32(D)))
        assert n == _fp64_recount(win, float(np.float32(D))), float(D)
        counts.append(n)
    assert sum(counts) > 0 and max(counts) <= 4


# ------------------------------------------------------------- arguments

def test_rejects_bad_arguments(oracle_lib):
    ok = O.Window(20, 20, 10.0, 10.0, [1], [2], [0.25], 0.0, 0.5)
    assert O.validate(ok, -1.0, 1.0) == 0
    assert O.validate(ok, -1.0, 1.6) != 0                 # D tau > 3/4
    assert O.validate(ok, 0.5, 0.4) != 0                  # empty interval
    assert O.validate(ok, float("nan"), 0.4) != 0
    assert O.validate(O.Window(20, 20, 10.0, 10.0, [1], [2], [0.75], 0.0, 0.5), -1, 1) != 0  # t > tau
    assert O.validate(O.Window(20, 20, 10.0, 10.0, [1], [2], [float("nan")], 0.0, 0.5), -1, 1) != 0
    assert O.validate(O.Window(20, 20, 10.0, 10.0, [1], [2], [0.1], 0.2, 0.5), -1, 1) != 0  # t < t0
    assert O.validate(O.Window(20, 20, 10.0, 10.0, [1], [2], [0.1], 0.0, 0.0), -1, 1) != 0  # tau = 0
    assert O.validate(O.Window(20, 20, 30.0, 10.0, [1], [2], [0.1], 0.0, 0.5), -1, 1) != 0  # FOE out
    assert O.validate(O.Window(20, 20, 10.0, 10.0, [20], [2], [0.1], 0.0, 0.5), -1, 1) != 0  # x = W
    assert O.validate(O.Window(20, 20, 10.0, 10.0, [3], [-1], [0.1], 0.0, 0.5), -1, 1) != 0  # y < 0
    assert O.validate(O.Window(20, 20, 10.0, 10.0, [3], [20], [0.1], 0.0, 0.5), -1, 1) != 0  # y = H
    assert O.validate(O.Window(20, 20, 10.0, 10.0, [3], [2], [0.1], 0.0, 0.5, 0.6), -1, 1) != 0  # t_ref > tau
    assert O.validate(O.Window(20, 20, 10.0, 10.0, [3], [2], [0.1], 0.0, 0.5, -0.1), -1, 1) != 0  # t_ref < 0
    assert O.validate(ok, -128.5, 1.0) != 0               # D tau < -64
    # the boundaries themselves are inside: the FOE on the frame's corners,
    # the last row and column, events at both ends of the window, D tau at
    # 3/4 and -64, the warp to either end of the window
    for fx, fy in ((0.0, 0.0), (20.0, 20.0)):
        assert O.validate(O.Window(20, 20, fx, fy, [19, 0], [0, 19], [0.0, 0.5], 0.0, 0.5), -1, 1) == 0
    assert O.validate(O.Window(20, 20, 10.0, 10.0, [1], [2], [2.5], 2.0, 0.5), -128.0, 1.5) == 0
    for t_ref in (0.0, 0.5):
        assert O.validate(O.Window(20, 20, 10.0, 10.0, [1], [2], [0.25], 0.0, 0.5, t_ref), -1, 1) == 0
    empty = O.Window(20, 20, 10.0, 10.0, [], [], [], 0.0, 0.5)
    assert O.contrast(empty, 0.3)[:3] == (0, 0, 0)
    r = O.solve(empty, -1.0, 1.0, 1e-4, 0.0, 1)
    assert r["nodes_expanded"] == 0 and r["K_hat"] == 0
