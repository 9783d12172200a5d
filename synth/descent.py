"""Synthetic event windows of a camera in pure ventral descent.

Scene model (the setting of Sec. 3.2-3.3: a fronto-parallel plane, no
horizontal motion, constant vertical velocity inside a window): a scene point
seen at image position x0 at the window start moves radially about the focus
of expansion as

    x(t) = FOE + (x0 - FOE) / (1 - D t),

with D the divergence at the window start (positive while approaching).  Each
signal event samples one point at a random time and is rounded to the nearest
pixel centre; noise events are uniform in space and time.  A scene point is
brighter or darker than its surround with equal odds, and all its events carry
that polarity (+1 / -1); noise events draw theirs one by one.  Events are
returned sorted by time, as a camera emits them.

Every random number comes from the counter-based SplitMix64 stream in
``synth.rng``, addressed by (seed, stream, counter), so any window can be
regenerated from its seed alone.
"""
from dataclasses import dataclass, field
import math

import numpy as np

from .rng import stream_key, uniform01

_S_POINT, _S_TIME, _S_NOISE, _S_POL, _S_PARAM, _S_NOISE_POL = 1, 2, 3, 4, 5, 6
_MAX_ATTEMPTS = 64     # point redraws before giving up
_TRIES = 8             # time redraws per event before the point is redrawn


@dataclass
class Window:
    """One event window: SoA events plus the geometry they were made with."""
    W: int
    H: int
    foe_x: float
    foe_y: float
    x: np.ndarray          # int16 [N]
    y: np.ndarray          # int16 [N]
    t: np.ndarray          # float32 [N], in [t0, t0 + tau]
    p: np.ndarray          # int8 [N], +1 / -1 (read only by the per-polarity objective)
    t0: float
    tau: float
    D_true: float
    n_signal: int
    n_noise: int
    seed: int
    meta: dict = field(default_factory=dict)

    @property
    def n(self):
        return int(self.x.shape[0])


def _polarity(u):
    return np.where(u < 0.5, 1, -1).astype(np.int8)


def _signal(W, H, fx, fy, n_signal, n_points, D, tau, seed):
    if n_signal == 0:
        return (np.zeros(0, np.int16),) * 2 + (np.zeros(0, np.float32), np.zeros(0, np.int8))
    n_points = max(1, min(n_points, n_signal))
    base, extra = divmod(n_signal, n_points)
    e_max = base + (1 if extra else 0)
    counts = np.full(n_points, base, np.int64)
    counts[:extra] += 1
    kp, kt = stream_key(seed, _S_POINT), stream_key(seed, _S_TIME)
    tau32 = np.float32(tau)

    xs = np.zeros((n_points, e_max), np.int64)
    ys = np.zeros((n_points, e_max), np.int64)
    ts = np.zeros((n_points, e_max), np.float32)
    pending = np.arange(n_points, dtype=np.int64)
    j = np.arange(e_max, dtype=np.int64)
    r = np.arange(_TRIES, dtype=np.int64)
    for a in range(_MAX_ATTEMPTS):
        if pending.size == 0:
            break
        pa = pending * _MAX_ATTEMPTS + a
        x0 = uniform01(kp, (2 * pa).astype(np.uint64)) * W
        y0 = uniform01(kp, (2 * pa + 1).astype(np.uint64)) * H
        ctr = ((pa[:, None, None] * e_max + j[None, :, None]) * _TRIES + r[None, None, :])
        t = (uniform01(kt, ctr.astype(np.uint64)) * float(tau32)).astype(np.float32)
        t = np.minimum(t, tau32)
        td = t.astype(np.float64)
        den = 1.0 - D * td
        px = np.floor(fx + (x0[:, None, None] - fx) / den + 0.5)
        py = np.floor(fy + (y0[:, None, None] - fy) / den + 0.5)
        ok = (px >= 0) & (px < W) & (py >= 0) & (py < H)
        first = np.argmax(ok, axis=2)                       # first in-frame try
        has = ok.any(axis=2) | (j[None, :] >= counts[pending][:, None])
        good = has.all(axis=1)
        gi = pending[good]
        sel = first[good]
        xs[gi] = np.take_along_axis(px[good], sel[..., None], axis=2)[..., 0]
        ys[gi] = np.take_along_axis(py[good], sel[..., None], axis=2)[..., 0]
        ts[gi] = np.take_along_axis(t[good], sel[..., None], axis=2)[..., 0]
        pending = pending[~good]
    if pending.size:
        raise RuntimeError("synthetic scene: %d points never fit in the frame" % pending.size)
    mask = j[None, :] < counts[:, None]
    pol = _polarity(uniform01(stream_key(seed, _S_POL), np.arange(n_points, dtype=np.uint64)))
    return xs[mask].astype(np.int16), ys[mask].astype(np.int16), ts[mask], np.repeat(pol, counts)


def make_window(W, H, foe_x, foe_y, n_signal, n_points, n_noise, D, tau, seed, t0=0.0):
    """Generate one window; see the module docstring for the model."""
    if not (1.0 - D * tau > 0.0):
        raise ValueError("D*tau must stay below 1")
    sx, sy, st, sp = _signal(W, H, float(foe_x), float(foe_y), int(n_signal), int(n_points), float(D),
                             float(tau), seed)
    kn = stream_key(seed, _S_NOISE)
    c = np.arange(int(n_noise), dtype=np.uint64)
    nx = np.minimum(np.floor(uniform01(kn, 3 * c) * W), W - 1).astype(np.int16)
    ny = np.minimum(np.floor(uniform01(kn, 3 * c + 1) * H), H - 1).astype(np.int16)
    tau32 = np.float32(tau)
    nt = np.minimum((uniform01(kn, 3 * c + 2) * float(tau32)).astype(np.float32), tau32)
    npol = _polarity(uniform01(stream_key(seed, _S_NOISE_POL), c))
    x = np.concatenate([sx, nx])
    y = np.concatenate([sy, ny])
    t = np.concatenate([st, nt])
    p = np.concatenate([sp, npol])
    order = np.argsort(t, kind="stable")
    x, y, t, p = x[order], y[order], t[order], p[order]
    if t0 != 0.0:
        t = (t.astype(np.float64) + t0).astype(np.float32)
    return Window(W=W, H=H, foe_x=float(foe_x), foe_y=float(foe_y), x=np.ascontiguousarray(x),
                  y=np.ascontiguousarray(y), t=np.ascontiguousarray(t), p=p, t0=float(t0),
                  tau=float(np.float32(tau)), D_true=float(D), n_signal=int(n_signal),
                  n_noise=int(n_noise), seed=int(seed))


# ----------------------------------------------------------------- workloads

def window_config1(seed=1000):
    """346x260, FOE (173,130), 150 points x 20 events + 1,000 noise, D=0.2, tau=0.5."""
    return make_window(346, 260, 173.0, 130.0, 3000, 150, 1000, 0.2, 0.5, seed)


def window_config2(seed=2000):
    """640x480, FOE (320,240), 100,000 events (30% noise), 2,000 points, D=0.35, tau=0.3."""
    return make_window(640, 480, 320.0, 240.0, 70000, 2000, 30000, 0.35, 0.3, seed)


def batch_params3(n_windows=256, seed=3000):
    """Per-window (N, D, noise fraction, tau) of the 256-window batch."""
    k = stream_key(seed, _S_PARAM)
    c = np.arange(n_windows, dtype=np.uint64) * np.uint64(4)
    n = np.floor(np.exp(math.log(5e3) + uniform01(k, c) * (math.log(2e5) - math.log(5e3)))).astype(np.int64)
    D = 0.05 + uniform01(k, c + np.uint64(1)) * 0.75
    noise = 0.1 + uniform01(k, c + np.uint64(2)) * 0.3
    tau = 0.1 + uniform01(k, c + np.uint64(3)) * 0.4
    return n, D, noise, tau


def batch_spec3(i, params, seed=3000, W=640, H=480):
    """make_window arguments of window i of the uneven batch."""
    n, D, noise, tau = params
    N = int(n[i])
    n_noise = int(round(N * float(noise[i])))
    n_sig = N - n_noise
    return (W, H, W / 2.0, H / 2.0, n_sig, max(1, n_sig // 35), n_noise, float(D[i]), float(tau[i]), seed + 1 + i)


def batch_window3(i, params, seed=3000, W=640, H=480):
    return make_window(*batch_spec3(i, params, seed, W, H))


def batch_config3(n_windows=256, seed=3000):
    """Windows of the uneven batch: 640x480, N log-uniform in [5k, 200k]."""
    params = batch_params3(n_windows, seed)
    return [batch_window3(i, params, seed) for i in range(n_windows)]


def batch_params4(n_windows, seed):
    """Per-window (N, D, noise fraction, tau) of warm-start training or
    evaluation windows: as the uneven batch, with N log-uniform in [20k, 100k]."""
    k = stream_key(seed, _S_PARAM)
    c = np.arange(n_windows, dtype=np.uint64) * np.uint64(4)
    n = np.floor(np.exp(math.log(2e4) + uniform01(k, c) * (math.log(1e5) - math.log(2e4)))).astype(np.int64)
    D = 0.05 + uniform01(k, c + np.uint64(1)) * 0.75
    noise = 0.1 + uniform01(k, c + np.uint64(2)) * 0.3
    tau = 0.1 + uniform01(k, c + np.uint64(3)) * 0.4
    return n, D, noise, tau


# Seed bases of the warm-start windows: training and held-out evaluation sets
# are disjoint from each other and from every other workload's seeds.
WARM_TRAIN_SEED = 20_000_000
WARM_EVAL_SEED = 10_000_000


def serve_spec5(stream, w, n_scale=1.0):
    """make_window arguments of window w (t_w = 0.1 w) of descent `stream` at
    1280x720: D = 1/(20 - t_w); N rises linearly with D from 50k (D=0.05) to
    1M (D=1.0); 15% noise; tau=0.2.  `n_scale` shrinks N for small cases."""
    tw = 0.1 * w
    D = 1.0 / (20.0 - tw)
    N = int((50_000 + (1_000_000 - 50_000) * (D - 0.05) / 0.95) * n_scale)
    n_noise = int(round(0.15 * N))
    n_sig = N - n_noise
    return (1280, 720, 640.0, 360.0, n_sig, max(1, n_sig // 35), n_noise, D, 0.2, 5000 + 1000 * stream + w)


def stream_slot_spec5(stream, k, n_scale=1.0):
    """make_window arguments and start time of 0.1 s slot k of descent
    `stream` as one continuous event stream: the serving descent's model at
    t_k = 0.1 k (D = 1/(20 - t_k)), half the events of a 0.2 s window.  A
    scene point of the slot moves as in the descent from t_k on, so
    consecutive slots continue one constant-velocity descent."""
    tk = 0.1 * k
    D = 1.0 / (20.0 - tk)
    N = int((50_000 + (1_000_000 - 50_000) * (D - 0.05) / 0.95) * n_scale) // 2
    n_noise = int(round(0.15 * N))
    n_sig = N - n_noise
    return (1280, 720, 640.0, 360.0, n_sig, max(1, n_sig // 35), n_noise, D, 0.1, 7_000_000 + 1000 * stream + k), tk


def stream_events5(stream, k0, k1, n_scale=1.0, with_polarity=False):
    """numpy (x, y, t) of slots k0..k1-1 of descent `stream`, sorted by time
    (and their polarities p as a fourth array with with_polarity=True)."""
    xs, ys, ts, ps = [], [], [], []
    for k in range(k0, k1):
        spec, tk = stream_slot_spec5(stream, k, n_scale)
        w = make_window(*spec, t0=tk)
        xs.append(w.x)
        ys.append(w.y)
        ts.append(w.t)
        ps.append(w.p)
    x, y, t, p = np.concatenate(xs), np.concatenate(ys), np.concatenate(ts), np.concatenate(ps)
    o = np.argsort(t, kind="stable")
    return (x[o], y[o], t[o], p[o]) if with_polarity else (x[o], y[o], t[o])


def serve_config5(stream, w, n_scale=1.0):
    """Window w of descent `stream` of the serving workload (serve_spec5)."""
    return make_window(*serve_spec5(stream, w, n_scale))
