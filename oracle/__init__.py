"""CPU oracle (plain C, loaded through ctypes) for the divergence estimator.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and the benchmark's CPU-baseline / reference leg may import this package.
The product path (``paper_2209_13168_gb300``) never imports it and shares no
code with it.

What each function follows (paper: McLeod et al., arXiv 2209.13168):
  warp_cells      Eq. (11), binary32, fixed operation order
  scale, scale_interval  the warp scale and the bound's widened scale range
  contrast        Eqs. (12)-(13) as the integer key K = M*S - N_in^2 = M^2 C
  bound           Eqs. (14)-(19) as Kbar = M*Sbar - N_full^2 >= K(D)
  solve           Algorithm 1 (pop-K rounds; K_pop = 1 is Algorithm 1 itself),
                  optionally warm-started from a guess D_warm +- w_warm
  features        the warm start's 16 radial x 8 temporal count histogram
  mlp_forward_f32 the warm start network in binary32, the device's order
  mlp_forward_f64, mlp_loss_f64  the same network in binary64, its training
                  loss and backprop gradient
  warm_map        network outputs -> (D_warm, w_warm)
  resample        the paper's fast mode: coordinates scaled to a coarser frame,
                  a random share of the events kept
  grid_max        exhaustive dense grid (brute force)
  sweep_max       exact breakpoint sweep (brute force)
  fp64_disagreements  the same warp in binary64, diagnostic only

Every function is pinned by tests/test_oracle_*.py against closed forms,
invariants and brute force; none is marked "parity unpinned".
tests/test_oracle_mutants.py plants plausible mistakes in copies of
oracle.c and checks that the pins catch each one.
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC"]


def build(force=False):
    """Compile oracle.c into liboracle.so next to it (gcc, no FMA contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h"))):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    subprocess.check_call(["gcc"] + CFLAGS + ["-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


class _Win(ctypes.Structure):
    _fields_ = [("W", ctypes.c_int32), ("H", ctypes.c_int32), ("foe_x", ctypes.c_float),
                ("foe_y", ctypes.c_float), ("x", ctypes.c_void_p), ("y", ctypes.c_void_p),
                ("t", ctypes.c_void_p), ("n", ctypes.c_int64), ("t0", ctypes.c_float),
                ("tau", ctypes.c_float), ("t_ref", ctypes.c_float), ("p", ctypes.c_void_p)]


class _I128(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_uint64), ("hi", ctypes.c_int64)]

    def value(self):
        return (int(self.hi) << 64) | int(self.lo)


class _Res(ctypes.Structure):
    _fields_ = [("D_star", ctypes.c_float), ("D_end", ctypes.c_float), ("contrast", ctypes.c_double),
                ("bound_gap", ctypes.c_double), ("K_hat", _I128), ("gap_K", _I128),
                ("nodes_expanded", ctypes.c_int64), ("point_evals", ctypes.c_int64),
                ("bound_evals", ctypes.c_int64), ("event_warps", ctypes.c_int64),
                ("cell_increments", ctypes.c_int64), ("bound_increments", ctypes.c_int64),
                ("rounds", ctypes.c_int64),
                ("max_queue", ctypes.c_int64), ("status", ctypes.c_int32)]


class _Rec(ctypes.Structure):
    _fields_ = [("D_lo", ctypes.c_float), ("D_hi", ctypes.c_float), ("D_c", ctypes.c_float),
                ("leaf", ctypes.c_int32), ("Kbar", _I128), ("K_c", _I128)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.POINTER
        L.or_validate.argtypes = [P(_Win), ctypes.c_float, ctypes.c_float]
        L.or_warp_cells.argtypes = [P(_Win), ctypes.c_float, ctypes.c_void_p, ctypes.c_void_p]
        L.or_warp_cells.restype = None
        L.or_fp64_disagreements.argtypes = [P(_Win), ctypes.c_float]
        L.or_fp64_disagreements.restype = ctypes.c_int64
        L.or_scale.argtypes = [ctypes.c_float, ctypes.c_float, ctypes.c_float]
        L.or_scale.restype = ctypes.c_float
        L.or_scale_interval.argtypes = [ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                        P(ctypes.c_float), P(ctypes.c_float)]
        L.or_scale_interval.restype = None
        L.or_contrast.argtypes = [P(_Win), ctypes.c_float, P(_I128), P(ctypes.c_uint64),
                                  P(ctypes.c_int64), ctypes.c_void_p]
        L.or_bound.argtypes = [P(_Win), ctypes.c_float, ctypes.c_float, P(_I128), P(ctypes.c_uint64),
                               P(ctypes.c_int64), ctypes.c_void_p]
        L.or_solve.argtypes = [P(_Win), ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_double,
                               ctypes.c_int32, P(_Res), ctypes.c_void_p, ctypes.c_int64,
                               P(ctypes.c_int64)]
        L.or_solve_warm.argtypes = [P(_Win), ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_double,
                                    ctypes.c_int32, ctypes.c_int32, ctypes.c_float, ctypes.c_float, P(_Res),
                                    ctypes.c_void_p, ctypes.c_int64, P(ctypes.c_int64)]
        L.or_features.argtypes = [P(_Win), ctypes.c_void_p, ctypes.c_void_p]
        L.or_mlp_forward_f32.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        L.or_mlp_forward_f32.restype = None
        L.or_mlp_forward_f64.argtypes = [ctypes.c_void_p] * 5
        L.or_mlp_forward_f64.restype = None
        L.or_mlp_loss_f64.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                      ctypes.c_void_p]
        L.or_mlp_loss_f64.restype = ctypes.c_double
        L.or_warm_map.argtypes = [ctypes.c_float, ctypes.c_float, ctypes.c_float, P(ctypes.c_float),
                                  P(ctypes.c_float)]
        L.or_warm_map.restype = None
        L.or_resample.argtypes = [P(_Win), ctypes.c_int32, ctypes.c_int32, ctypes.c_float, ctypes.c_uint64,
                                  ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        L.or_resample.restype = ctypes.c_int64
        L.or_resample_foe.argtypes = [P(_Win), ctypes.c_int32, ctypes.c_int32, P(ctypes.c_float), P(ctypes.c_float)]
        L.or_resample_foe.restype = None
        L.or_grid_max.argtypes = [P(_Win), ctypes.c_float, ctypes.c_float, ctypes.c_float, P(_I128),
                                  P(ctypes.c_float), P(ctypes.c_int64)]
        L.or_sweep_max.argtypes = [P(_Win), ctypes.c_float, ctypes.c_float, P(_I128), P(ctypes.c_float),
                                   P(ctypes.c_int64)]
        _lib = L
    return _lib


class OracleError(RuntimeError):
    pass


def _check(rc):
    if rc != 0:
        raise OracleError("oracle returned %d" % rc)


class Window:
    """Keeps the SoA arrays alive and exposes the C struct."""

    def __init__(self, W, H, foe_x, foe_y, x, y, t, t0=0.0, tau=0.5, t_ref=None, p=None):
        """t_ref: the time (since t0) the warp maps events to; None = tau (the paper's).
        p: event polarities (int8) for the per-polarity objective; None = unused."""
        self.x = np.ascontiguousarray(x, dtype=np.int16)
        self.y = np.ascontiguousarray(y, dtype=np.int16)
        self.t = np.ascontiguousarray(t, dtype=np.float32)
        self.p = None if p is None else np.ascontiguousarray(p, dtype=np.int8)
        self.W, self.H = int(W), int(H)
        self.planes = 1 if p is None else 2
        self.c = _Win(int(W), int(H), float(foe_x), float(foe_y), self.x.ctypes.data,
                      self.y.ctypes.data, self.t.ctypes.data, int(self.x.size), float(t0), float(tau),
                      float(np.float32(tau)) if t_ref is None else float(t_ref),
                      None if p is None else self.p.ctypes.data)

    @classmethod
    def of(cls, w, t_ref=None, polarity=False):
        """From a synth.Window; polarity=True uses its polarities."""
        return cls(w.W, w.H, w.foe_x, w.foe_y, w.x, w.y, w.t, w.t0, w.tau, t_ref, w.p if polarity else None)

    @property
    def M(self):
        return self.W * self.H

    def image(self, img):
        """A flat image buffer as [H][W], or [2][H][W] with polarity planes."""
        return img.reshape(self.H, self.W) if self.planes == 1 else img.reshape(2, self.H, self.W)


def validate(win, D_lo, D_hi):
    return lib().or_validate(ctypes.byref(win.c), D_lo, D_hi)


def warp_cells(win, D):
    ux = np.zeros(win.x.size, np.int32)
    uy = np.zeros(win.x.size, np.int32)
    lib().or_warp_cells(ctypes.byref(win.c), D, ux.ctypes.data, uy.ctypes.data)
    return ux, uy


def fp64_disagreements(win, D):
    return int(lib().or_fp64_disagreements(ctypes.byref(win.c), D))


def scale(D, t_rel, tau):
    """The binary32 warp scale s(D) = (1 - D t)/(1 - D tau) of Eq. (11)."""
    return float(lib().or_scale(D, t_rel, tau))


def scale_interval(D_lo, D_hi, t_rel, tau):
    """The widened scale interval [s_a, s_b] the bound uses for one event."""
    a, b = ctypes.c_float(), ctypes.c_float()
    lib().or_scale_interval(D_lo, D_hi, t_rel, tau, ctypes.byref(a), ctypes.byref(b))
    return a.value, b.value


def contrast(win, D, want_iwe=False):
    """(K, S, N_in, iwe-or-None) at hypothesis D."""
    k, s, n = _I128(), ctypes.c_uint64(), ctypes.c_int64()
    img = np.zeros(win.planes * win.M, np.uint32) if want_iwe else None
    _check(lib().or_contrast(ctypes.byref(win.c), D, ctypes.byref(k), ctypes.byref(s), ctypes.byref(n),
                             img.ctypes.data if want_iwe else None))
    return k.value(), int(s.value), int(n.value), (win.image(img) if want_iwe else None)


def bound(win, D_lo, D_hi, want_iwe=False):
    """(Kbar, Sbar, N_full, iwe-or-None) over [D_lo, D_hi]."""
    k, s, n = _I128(), ctypes.c_uint64(), ctypes.c_int64()
    img = np.zeros(win.planes * win.M, np.uint32) if want_iwe else None
    _check(lib().or_bound(ctypes.byref(win.c), D_lo, D_hi, ctypes.byref(k), ctypes.byref(s),
                          ctypes.byref(n), img.ctypes.data if want_iwe else None))
    return k.value(), int(s.value), int(n.value), (win.image(img) if want_iwe else None)


def solve(win, D_lo=-1.0, D_hi=1.0, tol_D=1e-4, gamma=0.0, K_pop=1, trace_cap=0, warm=None):
    """Algorithm 1; warm = (D_warm, w_warm) starts it from a guess."""
    r = _Res()
    tr = (_Rec * trace_cap)() if trace_cap else None
    tl = ctypes.c_int64(0)
    wf, wd, ww = (0, 0.0, 0.0) if warm is None else (1, float(warm[0]), float(warm[1]))
    _check(lib().or_solve_warm(ctypes.byref(win.c), D_lo, D_hi, tol_D, gamma, K_pop, wf, wd, ww, ctypes.byref(r),
                               ctypes.cast(tr, ctypes.c_void_p) if tr is not None else None, trace_cap,
                               ctypes.byref(tl)))
    out = {f: getattr(r, f) for f, _ in _Res._fields_ if f not in ("K_hat", "gap_K")}
    out["K_hat"] = r.K_hat.value()
    out["gap_K"] = r.gap_K.value()
    if tr is not None:
        n = min(tl.value, trace_cap)
        out["trace"] = [(tr[i].D_lo, tr[i].D_hi, tr[i].D_c, tr[i].leaf, tr[i].Kbar.value(), tr[i].K_c.value())
                        for i in range(n)]
        out["trace_len"] = tl.value
    return out


def grid_max(win, D_lo, D_hi, h):
    k, d, n = _I128(), ctypes.c_float(), ctypes.c_int64()
    _check(lib().or_grid_max(ctypes.byref(win.c), D_lo, D_hi, h, ctypes.byref(k), ctypes.byref(d),
                             ctypes.byref(n)))
    return k.value(), d.value, n.value


def sweep_max(win, D_lo, D_hi):
    k, d, n = _I128(), ctypes.c_float(), ctypes.c_int64()
    _check(lib().or_sweep_max(ctypes.byref(win.c), D_lo, D_hi, ctypes.byref(k), ctypes.byref(d),
                              ctypes.byref(n)))
    return k.value(), d.value, n.value


# ------------------------------------------------------ learned warm start
N_FEATURES = 128
N_HIDDEN = 128
N_PARAMS = 128 * 128 + 128 + 128 * 128 + 128 + 2 * 128 + 2
# offsets of W1 b1 W2 b2 W3 b3 in the parameter vector ([out][in] matrices)
OFFSETS = {"W1": 0, "b1": 16384, "W2": 16512, "b2": 32896, "W3": 33024, "b3": 33280}


def features(win):
    """(features float32[128], counts int64[128]); bin index = 8 * radial + temporal,
    feature = 128 * count / n."""
    f = np.zeros(N_FEATURES, np.float32)
    c = np.zeros(N_FEATURES, np.int64)
    _check(lib().or_features(ctypes.byref(win.c), f.ctypes.data, c.ctypes.data))
    return f, c


def mlp_forward_f32(params, x):
    p = np.ascontiguousarray(params, np.float32)
    x = np.ascontiguousarray(x, np.float32)
    o = np.zeros(2, np.float32)
    lib().or_mlp_forward_f32(p.ctypes.data, x.ctypes.data, o.ctypes.data)
    return o


def mlp_forward_f64(params, x):
    """(h1, h2, out) in binary64."""
    p = np.ascontiguousarray(params, np.float64)
    x = np.ascontiguousarray(x, np.float64)
    h1, h2, o = np.zeros(N_HIDDEN), np.zeros(N_HIDDEN), np.zeros(2)
    lib().or_mlp_forward_f64(p.ctypes.data, x.ctypes.data, h1.ctypes.data, h2.ctypes.data, o.ctypes.data)
    return h1, h2, o


def mlp_loss_f64(params, X, u_star, want_grad=True):
    """(mean loss, gradient or None) over the samples X[B][128] with targets u_star[B]."""
    p = np.ascontiguousarray(params, np.float64)
    X = np.ascontiguousarray(X, np.float64).reshape(-1, N_FEATURES)
    u = np.ascontiguousarray(u_star, np.float64)
    g = np.zeros(N_PARAMS) if want_grad else None
    loss = lib().or_mlp_loss_f64(p.ctypes.data, X.ctypes.data, u.ctypes.data, X.shape[0],
                                 g.ctypes.data if want_grad else None)
    return float(loss), g


def warm_map(u, l, tau):
    """(D_warm, w_warm) from the network outputs (u = D tau guess, l = log half-width)."""
    d, w = ctypes.c_float(), ctypes.c_float()
    lib().or_warm_map(u, l, tau, ctypes.byref(d), ctypes.byref(w))
    return d.value, w.value


def resample(win, W2, H2, keep, seed):
    """The fast mode's window: (Window on W2 x H2 with the scaled FOE)."""
    n = win.x.size
    x2 = np.zeros(max(n, 1), np.int16)
    y2 = np.zeros(max(n, 1), np.int16)
    t2 = np.zeros(max(n, 1), np.float32)
    m = lib().or_resample(ctypes.byref(win.c), W2, H2, keep, seed, x2.ctypes.data, y2.ctypes.data, t2.ctypes.data)
    fx, fy = ctypes.c_float(), ctypes.c_float()
    lib().or_resample_foe(ctypes.byref(win.c), W2, H2, ctypes.byref(fx), ctypes.byref(fy))
    return Window(W2, H2, fx.value, fy.value, x2[:m], y2[:m], t2[:m], win.c.t0, win.c.tau, win.c.t_ref)
