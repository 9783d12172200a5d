"""Pins of the oracle's learned warm start: features, network, loss, mapping,
and the warm-started search.

As for the rest of the oracle, nothing here compares it with itself: the
features against exact integer / rational binning, the binary64 network
against a hand-built network with a closed-form output and its gradient
against central finite differences, the binary32 network against the
binary64 one, and the warm-started search against the exhaustive
breakpoint sweep and against the plain search it must reduce to.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from synth import window_config1


def window(W, H, foe, x, y, t, tau=0.5, t0=0.0):
    return O.Window(W, H, foe[0], foe[1], np.asarray(x, np.int16), np.asarray(y, np.int16),
                    np.asarray(t, np.float32), t0, tau)


def tiny(seed, W=29, H=23, n=120, tau=0.5, foe=(14.0, 11.0)):
    rng = np.random.default_rng(seed)
    return window(W, H, foe, rng.integers(0, W, n), rng.integers(0, H, n),
                  (rng.random(n) * tau).astype(np.float32), tau)


def bf16_round(a):
    """Round float32 values to bfloat16 (nearest, ties to even), as float32."""
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def random_params(seed, scale=1.0):
    rng = np.random.default_rng(seed)
    p = np.zeros(O.N_PARAMS, np.float32)
    o = O.OFFSETS
    p[o["W1"]:o["b1"]] = rng.normal(0, scale * math.sqrt(2 / 128), 128 * 128)
    p[o["b1"]:o["W2"]] = rng.normal(0, 0.05, 128)
    p[o["W2"]:o["b2"]] = rng.normal(0, scale * math.sqrt(2 / 128), 128 * 128)
    p[o["b2"]:o["W3"]] = rng.normal(0, 0.05, 128)
    p[o["W3"]:o["b3"]] = rng.normal(0, math.sqrt(1 / 128), 256)
    p[o["b3"]:] = rng.normal(0, 0.1, 2)
    for k in ("W1", "W2", "W3"):
        sl = slice(o[k], o[k] + (256 if k == "W3" else 16384))
        p[sl] = bf16_round(p[sl])
    return p


# ---------------------------------------------------------------- features

def test_feature_counts_cover_every_event(oracle_lib):
    for seed in range(5):
        win = tiny(seed, n=500)
        f, c = O.features(win)
        assert c.sum() == 500
        assert abs(float(f.astype(np.float64).sum()) - 128.0) < 1e-3
        assert np.array_equal(f[c == 1], np.full((c == 1).sum(), np.float32(128.0 / 500.0)))


def exact_bins(W, H, fx, fy, x, y, t, tau):
    """Exact radial / temporal bins (integer FOE; t0 = 0), or None where the
    real value lies within 1e-4 of a bin boundary (binary32 may go either
    way there)."""
    cx, cy = max(fx, W - 1 - fx), max(fy, H - 1 - fy)
    R2 = cx * cx + cy * cy
    r2 = (x - fx) ** 2 + (y - fy) ** 2
    v = 16.0 * math.sqrt(r2 / R2)
    rb = max(k for k in range(17) if k * k * R2 <= 256 * r2)
    if abs(v - round(v)) < 1e-4 and round(v) not in (0, 16):
        return None
    q = 8 * Fraction(float(t)) / Fraction(float(tau))
    tb = math.floor(q)
    if abs(float(q) - round(float(q))) < 1e-4 and round(float(q)) not in (0, 8):
        return None
    return min(rb, 15), min(tb, 7)


def test_feature_bins_match_exact_arithmetic(oracle_lib):
    rng = np.random.default_rng(5)
    for W, H, fx, fy in ((64, 48, 32, 24), (41, 37, 3, 30), (97, 13, 96, 0)):
        x = rng.integers(0, W, 800)
        y = rng.integers(0, H, 800)
        t = (rng.random(800) * 0.3).astype(np.float32)
        want = np.zeros(128, np.int64)
        keep = []
        for i in range(800):
            b = exact_bins(W, H, fx, fy, int(x[i]), int(y[i]), t[i], np.float32(0.3))
            if b is not None:
                want[b[0] * 8 + b[1]] += 1
                keep.append(i)
        assert len(keep) > 700
        keep = np.array(keep)
        _, c = O.features(window(W, H, (float(fx), float(fy)), x[keep], y[keep], t[keep], tau=0.3))
        assert np.array_equal(c, want)


def test_feature_special_cases(oracle_lib):
    # The FOE pixel is radial bin 0, the farthest corner bin 15 (r = R, clamped);
    # t = t0 is temporal bin 0, t = t0 + tau bin 7 (clamped).
    win = window(40, 30, (10.0, 20.0), [10, 39, 39, 10], [20, 0, 0, 20], [2.0, 2.0, 2.25, 2.25], tau=0.25,
                 t0=2.0)
    _, c = O.features(win)
    assert c[0 * 8 + 0] == 1 and c[15 * 8 + 0] == 1 and c[15 * 8 + 7] == 1 and c[0 * 8 + 7] == 1
    assert c.sum() == 4
    f, c = O.features(window(40, 30, (10.0, 20.0), [], [], [], tau=0.25))
    assert c.sum() == 0 and not f.any()


# ----------------------------------------------------------------- network

def test_network_closed_form(oracle_lib):
    # W1 = W2 = identity, zero hidden biases, W3 = [ones; e_0]: the hidden
    # layers pass relu(x) through, so out0 = sum(relu(x)) + b3[0] and
    # out1 = relu(x0) + b3[1].
    o = O.OFFSETS
    p = np.zeros(O.N_PARAMS)
    p[o["W1"]:o["b1"]] = np.eye(128).ravel()
    p[o["W2"]:o["b2"]] = np.eye(128).ravel()
    p[o["W3"]:o["W3"] + 128] = 1.0
    p[o["W3"] + 128] = 1.0
    p[o["b3"]:] = [0.25, -0.5]
    x = np.random.default_rng(1).normal(0, 1, 128)
    h1, h2, out = O.mlp_forward_f64(p, x)
    r = np.maximum(x, 0)
    assert np.allclose(h1, r, rtol=0, atol=0) and np.allclose(h2, r, rtol=0, atol=0)
    assert out[0] == pytest.approx(r.sum() + 0.25, rel=1e-15)
    assert out[1] == pytest.approx(r[0] - 0.5, rel=1e-15)
    o32 = O.mlp_forward_f32(p.astype(np.float32), x.astype(np.float32))
    assert o32[0] == pytest.approx(r.sum() + 0.25, rel=1e-6)


def test_loss_gradient_matches_finite_differences(oracle_lib):
    rng = np.random.default_rng(7)
    p = random_params(3).astype(np.float64)
    X = rng.random((6, 128)) * 2
    u = rng.uniform(0.0, 0.4, 6)
    loss, g = O.mlp_loss_f64(p, X, u)
    o = O.OFFSETS
    idx = list(rng.choice(o["b1"], 60, replace=False)) + list(range(o["b1"], o["b1"] + 20))
    idx += list(o["W2"] + rng.choice(16384, 60, replace=False)) + list(range(o["b2"], o["b2"] + 20))
    idx += list(range(o["W3"], o["W3"] + 256, 5)) + [o["b3"], o["b3"] + 1]
    h = 1e-6
    for i in idx:
        q = p.copy()
        q[i] += h
        lp, _ = O.mlp_loss_f64(q, X, u, want_grad=False)
        q[i] -= 2 * h
        lm, _ = O.mlp_loss_f64(q, X, u, want_grad=False)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])), (i, fd, g[i])


def test_loss_value_and_minimiser(oracle_lib):
    # With W3 = 0 the outputs are the biases: loss = 9/2 e^2 exp(-2 l) + l, whose
    # minimum over l for one sample is at exp(l) = 3 |e| (the half-width covers
    # three standard deviations).
    o = O.OFFSETS
    p = random_params(4).astype(np.float64)
    p[o["W3"]:o["b3"]] = 0.0
    X = np.random.default_rng(2).random((3, 128))
    for b in (-1.3, -6.0, 2.5):
        p[o["b3"]:] = [0.1, b]
        u = np.array([0.3, 0.1, 0.2])
        loss, g = O.mlp_loss_f64(p, X, u)
        e = u - 0.1
        want = np.mean(4.5 * e * e * math.exp(-2 * b) + b)
        assert loss == pytest.approx(want, rel=1e-12)
        assert g[o["b3"] + 1] == pytest.approx(np.mean(1 - 9 * e * e * math.exp(-2 * b)), rel=1e-12)
        assert g[o["b3"]] == pytest.approx(np.mean(-9 * e * math.exp(-2 * b)), rel=1e-12)
    p[o["b3"]:] = [0.1, math.log(3 * 0.05)]
    _, g = O.mlp_loss_f64(p, X[:1], np.array([0.15]))
    assert abs(g[o["b3"] + 1]) < 1e-12


def test_binary32_network_tracks_binary64(oracle_lib):
    # The device's binary32 evaluation order stays within 1e-3 (relative to
    # the output scale) of the binary64 network on the same bf16 weights.
    rng = np.random.default_rng(9)
    for s in range(8):
        p = random_params(10 + s)
        x = (rng.random(128) * 2).astype(np.float32)
        o32 = O.mlp_forward_f32(p, x).astype(np.float64)
        _, _, o64 = O.mlp_forward_f64(p.astype(np.float64), x.astype(np.float64))
        assert np.all(np.abs(o32 - o64) <= 1e-3 * np.maximum(np.abs(o64), 1e-2))


def test_warm_map(oracle_lib):
    tau = 0.3
    for k in range(-20, 2):
        D, w = O.warm_map(0.12, k * math.log(2.0), tau)
        assert w == np.float32(np.float32(2.0 ** k) / np.float32(tau))
        assert D == np.float32(np.float32(0.12) / np.float32(tau))
    for k in range(-12, 1):                       # the exponent rounds to nearest
        assert O.warm_map(0.0, (k + 0.4) * math.log(2.0), tau)[1] == np.float32(np.float32(2.0 ** k) / np.float32(tau))
        assert O.warm_map(0.0, (k + 0.6) * math.log(2.0), tau)[1] == np.float32(
            np.float32(2.0 ** (k + 1)) / np.float32(tau))
    assert O.warm_map(0.0, 50.0, tau)[1] == np.float32(np.float32(2.0) / np.float32(tau))
    assert O.warm_map(0.0, -50.0, tau)[1] == np.float32(np.float32(2.0 ** -20) / np.float32(tau))
    assert O.warm_map(0.0, float("nan"), tau)[1] == np.float32(np.float32(2.0 ** -20) / np.float32(tau))


# -------------------------------------------------------- warm-started search

def test_warm_start_covering_the_domain_is_the_plain_search(oracle_lib):
    # A guess at the centre with a half-width beyond the domain leaves one
    # piece, the domain itself, and the centre as incumbent: Algorithm 1
    # exactly, step for step.
    win = O.Window.of(window_config1())
    for K in (1, 8):
        a = O.solve(win, -1.0, 1.0, 1e-4, 0.0, K, trace_cap=4096)
        b = O.solve(win, -1.0, 1.0, 1e-4, 0.0, K, trace_cap=4096, warm=(0.0, 4.0))
        assert a == b


@pytest.mark.parametrize("K_pop", [1, 4])
def test_warm_start_agrees_with_brute_force(oracle_lib, K_pop):
    # Any guess, good, bad or outside the domain: the certificate still covers
    # the exhaustive maximum, and the incumbent is attained.
    rng = np.random.default_rng(41 + K_pop)
    for seed in range(6):
        W, H = int(rng.integers(10, 33)), int(rng.integers(10, 33))
        win = tiny(300 + seed, W=W, H=H, n=int(rng.integers(20, 200)), foe=(float(W // 2), float(H // 2)))
        Kmax, Dmax, _ = O.sweep_max(win, -1.0, 1.0)
        for g, hw in ((Dmax, 1e-3), (float(rng.uniform(-1, 1)), 0.05), (3.0, 0.25), (-1.0, 0.5), (Dmax, 2.0)):
            r = O.solve(win, -1.0, 1.0, 1e-4, 0.0, K_pop, warm=(g, hw))
            assert O.contrast(win, r["D_star"])[0] == r["K_hat"]
            assert r["K_hat"] <= Kmax <= r["K_hat"] + r["gap_K"]


def test_warm_start_pieces(oracle_lib):
    # The domain enters as the pieces [lo, g-w], [g-w, g+w], [g+w, hi] (those of
    # positive width): point evaluations = 1 + expansions and bound
    # evaluations = pieces + 2 per split expansion.
    win = O.Window.of(window_config1())
    for g, hw, pieces in ((0.3, 0.05, 3), (-1.0, 0.25, 2), (1.7, 0.25, 2), (0.0, 1.0, 1)):
        r = O.solve(win, -1.0, 1.0, 1e-4, 0.0, 1, trace_cap=8192, warm=(g, hw))
        splits = sum(1 for rec in r["trace"] if not rec[3])
        assert r["point_evals"] == 1 + r["nodes_expanded"]
        assert r["bound_evals"] == pieces + 2 * splits
        # the first expanded interval lies in one piece
        lo, hi = r["trace"][0][0], r["trace"][0][1]
        cuts = sorted({-1.0, 1.0, float(np.float32(max(-1.0, min(1.0, g)) - np.float32(hw))),
                       float(np.float32(max(-1.0, min(1.0, g)) + np.float32(hw)))})
        assert any(a <= lo and hi <= b for a, b in zip(cuts, cuts[1:]))


def test_warm_start_rejects_bad_guesses(oracle_lib):
    win = tiny(1)
    for g, hw in ((float("nan"), 0.1), (0.1, 0.0), (0.1, -1.0), (0.1, float("inf"))):
        with pytest.raises(O.OracleError):
            O.solve(win, -1.0, 1.0, 1e-4, 0.0, 1, warm=(g, hw))
