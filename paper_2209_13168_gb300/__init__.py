"""Python binding of libdd.so, the GB300 (sm_103a) exact divergence estimator.

Argument marshalling only: every step of the estimator (event ingest, warp,
IWE scatter, sums of squares, bounds, the branch-and-bound queue) runs in the
CUDA kernels behind include/dd.h.  There is no CPU fallback: if libdd.so is
missing or fails to load, every entry point raises.

The functions keep the C names (dd_create, dd_contrast, dd_bound, dd_solve,
dd_solve_trace, dd_solve_window, dd_solve_batch, dd_features, dd_set_warm_model,
dd_set_stream, dd_get_stats, dd_reset_stats, dd_set_timing, dd_destroy,
dd_strerror, dd_resample, dd_resample_foe, dd_time_span, dd_stream_solve,
dd_probe_peaks, the dd_serve_* and dd_mlp_* families); ``Context``, ``Server``
and ``Mlp`` wrap them for numpy arrays (host events) and torch CUDA tensors
(device events, features, training batches).

Window parameters are tuples (D_lo, D_hi, tol_D, gamma[, warm]) with warm
None (Algorithm 1 from the centre), "model" (the context's warm-start model)
or (D_warm, w_warm) (a given guess and half-width).
"""
import ctypes
import json
import os
import time

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libdd.so")

DD_OK, DD_ERR_ARG, DD_ERR_OOM, DD_ERR_QUEUE_OVERFLOW, DD_ERR_TIMEOUT, DD_ERR_CUDA, DD_ERR_NO_DEVICE = \
    0, -1, -2, -3, -4, -5, -6
DD_ERR_CAPACITY = -7
DD_ERR_CANCELLED = -8
DD_PENDING = 1
DD_NOALLOC_MAX_EVENTS = 1 << 20
DD_WARM_NONE, DD_WARM_GIVEN, DD_WARM_MODEL = 0, 1, 2
DD_MLP_FEATURES, DD_MLP_PARAMS = 128, 33282


class DDError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__("%s: %s (%d)" % (where, dd_strerror(status), status))


class dd_i128(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_uint64), ("hi", ctypes.c_int64)]

    def value(self):
        return (int(self.hi) << 64) | int(self.lo)


class dd_config(ctypes.Structure):
    _fields_ = [("pop_k", ctypes.c_int32), ("queue_capacity", ctypes.c_int32), ("band_rows", ctypes.c_int32),
                ("threads", ctypes.c_int32), ("max_rounds", ctypes.c_int32), ("host_loop", ctypes.c_int32),
                ("max_splits", ctypes.c_int32), ("warp_to_start", ctypes.c_int32), ("polarity", ctypes.c_int32),
                ("fuse_span", ctypes.c_int32)]


class dd_events(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("t", ctypes.c_void_p), ("n", ctypes.c_int64),
                ("t0", ctypes.c_float), ("tau", ctypes.c_float), ("device_ptrs", ctypes.c_int32),
                ("p", ctypes.c_void_p)]


class dd_result(ctypes.Structure):
    _fields_ = [("D_star", ctypes.c_float), ("D_end", ctypes.c_float), ("contrast", ctypes.c_double),
                ("bound_gap", ctypes.c_double), ("K_hat", dd_i128), ("gap_K", dd_i128),
                ("nodes_expanded", ctypes.c_int64), ("point_evals", ctypes.c_int64),
                ("bound_evals", ctypes.c_int64), ("event_warps", ctypes.c_int64),
                ("cell_increments", ctypes.c_int64), ("bound_increments", ctypes.c_int64),
                ("rounds", ctypes.c_int64), ("max_queue", ctypes.c_int64),
                ("status", ctypes.c_int32), ("D_warm", ctypes.c_float), ("w_warm", ctypes.c_float)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_ if f not in ("K_hat", "gap_K")}
        d["K_hat"] = self.K_hat.value()
        d["gap_K"] = self.gap_K.value()
        return d


class dd_window_params(ctypes.Structure):
    _fields_ = [("D_lo", ctypes.c_float), ("D_hi", ctypes.c_float), ("tol_D", ctypes.c_float),
                ("warm", ctypes.c_int32), ("gamma", ctypes.c_double), ("D_warm", ctypes.c_float),
                ("w_warm", ctypes.c_float)]


def window_params(p):
    """dd_window_params from (D_lo, D_hi, tol_D, gamma[, warm])."""
    warm = p[4] if len(p) > 4 else None
    if warm is None:
        return dd_window_params(p[0], p[1], p[2], DD_WARM_NONE, p[3], 0.0, 0.0)
    if isinstance(warm, str):
        if warm != "model":
            raise ValueError("warm must be None, 'model' or (D_warm, w_warm)")
        return dd_window_params(p[0], p[1], p[2], DD_WARM_MODEL, p[3], 0.0, 0.0)
    return dd_window_params(p[0], p[1], p[2], DD_WARM_GIVEN, p[3], float(warm[0]), float(warm[1]))


class dd_node_rec(ctypes.Structure):
    _fields_ = [("D_lo", ctypes.c_float), ("D_hi", ctypes.c_float), ("D_c", ctypes.c_float),
                ("leaf", ctypes.c_int32), ("Kbar", dd_i128), ("K_c", dd_i128)]


class dd_stats(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_int64), ("eval_launches", ctypes.c_int64),
                ("h2d_bytes", ctypes.c_int64), ("d2h_bytes", ctypes.c_int64), ("host_syncs", ctypes.c_int64),
                ("timed_launches", ctypes.c_int64), ("eval_ms", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


# Every symbol include/dd.h declares, with its ctypes signature.
_P = ctypes.POINTER
_VP = ctypes.c_void_p
SIGNATURES = {
    "dd_create": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_float, ctypes.c_float, _P(dd_config),
                                 _P(_VP)]),
    "dd_destroy": (None, [_VP]),
    "dd_set_stream": (ctypes.c_int, [_VP, _VP]),
    "dd_contrast": (ctypes.c_int, [_VP, _P(dd_events), _VP, ctypes.c_int32, _VP, _VP, _VP, _VP]),
    "dd_bound": (ctypes.c_int, [_VP, _P(dd_events), _VP, _VP, ctypes.c_int32, _VP, _VP, _VP, _VP]),
    "dd_solve": (ctypes.c_int, [_VP, _P(dd_events), ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_double,
                                _P(dd_result)]),
    "dd_solve_trace": (ctypes.c_int, [_VP, _P(dd_events), ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                      ctypes.c_double, _P(dd_result), _VP, ctypes.c_int64, _P(ctypes.c_int64)]),
    "dd_solve_batch": (ctypes.c_int, [_VP, _P(dd_events), ctypes.c_int32, _P(dd_window_params), _P(dd_result)]),
    "dd_solve_window": (ctypes.c_int, [_VP, _P(dd_events), _P(dd_window_params), _P(dd_result), _VP,
                                       ctypes.c_int64, _P(ctypes.c_int64)]),
    "dd_features": (ctypes.c_int, [_VP, _P(dd_events), ctypes.c_int32, _VP]),
    "dd_set_warm_model": (ctypes.c_int, [_VP, _VP]),
    "dd_mlp_create": (ctypes.c_int, [ctypes.c_uint64, _P(_VP)]),
    "dd_mlp_destroy": (None, [_VP]),
    "dd_mlp_set_stream": (ctypes.c_int, [_VP, _VP]),
    "dd_mlp_get_params": (ctypes.c_int, [_VP, _VP, ctypes.c_int64]),
    "dd_mlp_set_params": (ctypes.c_int, [_VP, _VP, ctypes.c_int64]),
    "dd_mlp_save": (ctypes.c_int, [_VP, ctypes.c_char_p]),
    "dd_mlp_load": (ctypes.c_int, [_VP, ctypes.c_char_p]),
    "dd_mlp_forward": (ctypes.c_int, [_VP, _VP, ctypes.c_int32, _VP]),
    "dd_mlp_grad": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int32, _VP, _VP]),
    "dd_mlp_train_step": (ctypes.c_int, [_VP, _VP, _VP, ctypes.c_int32, ctypes.c_float, _VP]),
    "dd_serve_start": (ctypes.c_int, [_VP, ctypes.c_int32, ctypes.c_int64, _P(_VP)]),
    "dd_serve_slots": (ctypes.c_int, [_VP, _P(ctypes.c_int32), _P(ctypes.c_int64)]),
    "dd_serve_submit": (ctypes.c_int, [_VP, _P(dd_events), _P(dd_window_params), ctypes.c_double,
                                       _P(ctypes.c_uint64)]),
    "dd_serve_poll": (ctypes.c_int, [_VP, ctypes.c_uint64, _P(dd_result), _P(ctypes.c_double)]),
    "dd_serve_cancel": (ctypes.c_int, [_VP, ctypes.c_uint64]),
    "dd_serve_wait": (ctypes.c_int, [_VP, ctypes.c_uint64, _P(dd_result), _P(ctypes.c_double)]),
    "dd_serve_stats": (ctypes.c_int, [_VP, _P(ctypes.c_int64), _P(ctypes.c_int64), _P(ctypes.c_int64)]),
    "dd_serve_stop": (ctypes.c_int, [_VP]),
    "dd_serve_clock": (ctypes.c_double, []),
    "dd_get_stats": (ctypes.c_int, [_VP, _P(dd_stats)]),
    "dd_reset_stats": (ctypes.c_int, [_VP]),
    "dd_set_timing": (ctypes.c_int, [_VP, ctypes.c_int32]),
    "dd_get_launch_times": (ctypes.c_int, [_VP, _VP, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    "dd_contrast_noalloc": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_float, ctypes.c_float,
                                           _P(dd_events), _VP, ctypes.c_int32, _VP, _VP]),
    "dd_probe_peaks": (ctypes.c_int, [_P(ctypes.c_double), _P(ctypes.c_double), _VP]),
    "dd_resample": (ctypes.c_int, [_VP, _P(dd_events), ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                   ctypes.c_int32, ctypes.c_float, ctypes.c_uint64, _VP, _VP, _VP,
                                   _P(ctypes.c_int64)]),
    "dd_stream_solve": (ctypes.c_int, [_VP, _P(dd_events), ctypes.c_double, ctypes.c_float, ctypes.c_double,
                                       ctypes.c_int32, _P(dd_window_params), _P(dd_result), _VP, _VP]),
    "dd_check_flags": (ctypes.c_int, [_P(ctypes.c_uint32), _P(ctypes.c_int32), ctypes.c_int32]),
    "dd_time_span": (ctypes.c_int, [_VP, ctypes.POINTER(dd_events), ctypes.POINTER(ctypes.c_float),
                                    ctypes.POINTER(ctypes.c_float)]),
    "dd_resample_foe": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_float, ctypes.c_float,
                                       ctypes.c_int32, ctypes.c_int32, _P(ctypes.c_float), _P(ctypes.c_float)]),
    "dd_strerror": (ctypes.c_char_p, [ctypes.c_int]),
}

_lib = None


def load(path=None):
    """Load libdd.so (built by __graft_entry__.build(); the environment
    variable DD_LIBRARY names another build, e.g. the checked one); raises if
    it is absent."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or os.environ.get("DD_LIBRARY") or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError("libdd.so not found at %s: build it with __graft_entry__.build() "
                           "(the estimator has no CPU fallback)" % p)
    L = ctypes.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def dd_strerror(status):
    return load().dd_strerror(int(status)).decode()


def _check(rc, where):
    if rc != DD_OK:
        raise DDError(rc, where)


def dd_create(W, H, foe_x, foe_y, cfg=None):
    h = _VP()
    _check(load().dd_create(W, H, foe_x, foe_y, ctypes.byref(cfg) if cfg is not None else None, ctypes.byref(h)),
           "dd_create")
    return h


def dd_destroy(h):
    load().dd_destroy(h)


def dd_set_stream(h, stream_ptr):
    _check(load().dd_set_stream(h, _VP(stream_ptr) if stream_ptr else None), "dd_set_stream")


def dd_get_stats(h):
    s = dd_stats()
    _check(load().dd_get_stats(h, ctypes.byref(s)), "dd_get_stats")
    return s.as_dict()


def dd_reset_stats(h):
    _check(load().dd_reset_stats(h), "dd_reset_stats")


def dd_set_timing(h, enable):
    _check(load().dd_set_timing(h, 1 if enable else 0), "dd_set_timing")


def dd_get_launch_times(h):
    """Device durations (ms) of the timed evaluation launches since the last reset."""
    n = ctypes.c_int32(0)
    _check(load().dd_get_launch_times(h, None, 0, ctypes.byref(n)), "dd_get_launch_times")
    ms = np.zeros(max(n.value, 1), np.float32)
    _check(load().dd_get_launch_times(h, ms.ctypes.data, n.value, ctypes.byref(n)), "dd_get_launch_times")
    return ms[:n.value]


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _host_ints(a, dtype, name):
    """A host array of integers as a contiguous array of `dtype`; values that
    are not integers or do not fit are an error, not a silent cast."""
    a = np.asarray(a)
    if a.ndim != 1:
        raise ValueError("%s: a 1-D array is required" % name)
    if a.dtype != dtype and a.size:
        info = np.iinfo(dtype)
        if a.dtype.kind not in "iu" and not np.all(np.equal(np.mod(a, 1), 0)):
            raise ValueError("%s: integer values are required" % name)
        if a.min() < info.min or a.max() > info.max:
            raise ValueError("%s: values outside %s" % (name, np.dtype(dtype).name))
    return np.ascontiguousarray(a, dtype=dtype)


class Events:
    """dd_events over numpy arrays (host) or torch CUDA tensors (device).

    Holds references to the arrays so they outlive the call."""

    def __init__(self, x, y, t, t0, tau, p=None):
        """p: int8 polarities (same kind of memory as x/y/t), read by a
        context with polarity=1; None otherwise.  Host arrays are converted
        (coordinates must be integers within int16, polarities within int8);
        CUDA tensors must already have the ABI's types."""
        dev = hasattr(x, "is_cuda") and x.is_cuda
        if dev:
            import torch
            want = ((x, torch.int16, "x"), (y, torch.int16, "y"), (t, torch.float32, "t")) + \
                (() if p is None else ((p, torch.int8, "p"),))
            for a, dt, name in want:
                if not (hasattr(a, "is_cuda") and a.is_cuda and a.dtype == dt and a.dim() == 1 and a.is_contiguous()):
                    raise TypeError("%s: a contiguous 1-D CUDA tensor of %s is required" % (name, dt))
        else:
            x = _host_ints(x, np.int16, "x")
            y = _host_ints(y, np.int16, "y")
            t = np.ascontiguousarray(t, dtype=np.float32)
            if t.ndim != 1:
                raise ValueError("t: a 1-D array is required")
            p = None if p is None else _host_ints(p, np.int8, "p")
        n = int(x.shape[0])
        if any(int(a.shape[0]) != n for a in (y, t) + (() if p is None else (p,))):
            raise ValueError("x, y, t (and p) must have the same length")
        self.x, self.y, self.t, self.p = x, y, t, p
        self.c = dd_events(_ptr(x) if n else None, _ptr(y) if n else None, _ptr(t) if n else None, n,
                           float(t0), float(tau), 1 if dev else 0, _ptr(p) if (n and p is not None) else None)

    def with_time(self, t0, tau):
        """The same arrays as a window [t0, t0 + tau] (e.g. from Context.time_span)."""
        return Events(self.x, self.y, self.t, t0, tau, self.p)

    @classmethod
    def of(cls, w, device=None, polarity=False):
        """From a synth.Window (numpy arrays, or torch CUDA tensors already on the
        device); device='cuda' uploads numpy arrays as torch tensors;
        polarity=True passes the window's polarities."""
        p = w.p if polarity else None
        if polarity and p is None:
            raise ValueError("the window has no polarities")
        if hasattr(w.x, "is_cuda") and w.x.is_cuda:
            return cls(w.x, w.y, w.t, w.t0, w.tau, p)
        if device is None:
            return cls(w.x, w.y, w.t, w.t0, w.tau, p)
        import torch
        return cls(torch.from_numpy(w.x).to(device), torch.from_numpy(w.y).to(device),
                   torch.from_numpy(w.t).to(device), w.t0, w.tau,
                   None if p is None else torch.from_numpy(p).to(device))


def dd_contrast(h, ev, D, want=("S", "N"), want_iwe=False, M=None):
    D = np.ascontiguousarray(D, dtype=np.float32)
    n = D.size
    K = (dd_i128 * max(n, 1))()
    S = np.zeros(n, np.uint64)
    N = np.zeros(n, np.int64)
    img = np.zeros(n * M, np.uint32) if want_iwe else None
    _check(load().dd_contrast(h, ctypes.byref(ev.c), D.ctypes.data, n, ctypes.cast(K, _VP), S.ctypes.data,
                              N.ctypes.data, img.ctypes.data if want_iwe else None), "dd_contrast")
    return [K[i].value() for i in range(n)], S, N, img


def dd_bound(h, ev, D_lo, D_hi, want_iwe=False, M=None):
    D_lo = np.ascontiguousarray(D_lo, dtype=np.float32)
    D_hi = np.ascontiguousarray(D_hi, dtype=np.float32)
    n = D_lo.size
    K = (dd_i128 * max(n, 1))()
    S = np.zeros(n, np.uint64)
    N = np.zeros(n, np.int64)
    img = np.zeros(n * M, np.uint32) if want_iwe else None
    _check(load().dd_bound(h, ctypes.byref(ev.c), D_lo.ctypes.data, D_hi.ctypes.data, n, ctypes.cast(K, _VP),
                           S.ctypes.data, N.ctypes.data, img.ctypes.data if want_iwe else None), "dd_bound")
    return [K[i].value() for i in range(n)], S, N, img


def dd_solve(h, ev, D_lo, D_hi, tol_D, gamma):
    r = dd_result()
    _check(load().dd_solve(h, ctypes.byref(ev.c), D_lo, D_hi, tol_D, gamma, ctypes.byref(r)), "dd_solve")
    return r.as_dict()


def dd_solve_batch(h, evs, params):
    """evs: list of Events; params: list of (D_lo, D_hi, tol_D, gamma).
    Returns (status, [result dicts]) when the windows ran (each result has its
    own status); raises when the call itself failed."""
    n = len(evs)
    E = (dd_events * n)(*[e.c for e in evs])
    P = (dd_window_params * n)(*[window_params(p) for p in params])
    R = (dd_result * n)()
    rc = load().dd_solve_batch(h, E, n, P, R)
    res = [R[i].as_dict() for i in range(n)]
    if rc != DD_OK and all(r["status"] == DD_OK for r in res):
        raise DDError(rc, "dd_solve_batch")      # the call itself failed
    return rc, res


def dd_solve_trace(h, ev, D_lo, D_hi, tol_D, gamma, trace_cap):
    r = dd_result()
    tr = (dd_node_rec * max(trace_cap, 1))()
    tl = ctypes.c_int64(0)
    _check(load().dd_solve_trace(h, ctypes.byref(ev.c), D_lo, D_hi, tol_D, gamma, ctypes.byref(r),
                                 ctypes.cast(tr, _VP), trace_cap, ctypes.byref(tl)), "dd_solve_trace")
    d = r.as_dict()
    d["trace"] = [(tr[i].D_lo, tr[i].D_hi, tr[i].D_c, tr[i].leaf, tr[i].Kbar.value(), tr[i].K_c.value())
                  for i in range(min(tl.value, trace_cap))]
    d["trace_len"] = tl.value
    return d


def dd_solve_window(h, ev, params, trace_cap=0):
    """One window with full parameters (warm start included), optional trace."""
    r = dd_result()
    p = window_params(params)
    tr = (dd_node_rec * max(trace_cap, 1))()
    tl = ctypes.c_int64(0)
    _check(load().dd_solve_window(h, ctypes.byref(ev.c), ctypes.byref(p), ctypes.byref(r),
                                  ctypes.cast(tr, _VP) if trace_cap else None, trace_cap, ctypes.byref(tl)),
           "dd_solve_window")
    d = r.as_dict()
    if trace_cap:
        d["trace"] = [(tr[i].D_lo, tr[i].D_hi, tr[i].D_c, tr[i].leaf, tr[i].Kbar.value(), tr[i].K_c.value())
                      for i in range(min(tl.value, trace_cap))]
        d["trace_len"] = tl.value
    return d


def dd_features(h, evs):
    """Warm-start features of the windows (list of Events): torch CUDA tensor [n][128]."""
    import torch
    n = len(evs)
    E = (dd_events * n)(*[e.c for e in evs])
    out = torch.empty((n, DD_MLP_FEATURES), dtype=torch.float32, device="cuda")
    _check(load().dd_features(h, E, n, out.data_ptr()), "dd_features")
    return out


class Mlp:
    """The warm-start network (dd_mlp_*); batches are torch CUDA tensors."""

    def __init__(self, seed=0, path=None):
        h = _VP()
        _check(load().dd_mlp_create(int(seed), ctypes.byref(h)), "dd_mlp_create")
        self.h = h
        if path:
            self.load(path)

    def close(self):
        if self.h:
            load().dd_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream_ptr):
        _check(load().dd_mlp_set_stream(self.h, _VP(stream_ptr) if stream_ptr else None), "dd_mlp_set_stream")

    def get_params(self):
        p = np.zeros(DD_MLP_PARAMS, np.float32)
        _check(load().dd_mlp_get_params(self.h, p.ctypes.data, p.size), "dd_mlp_get_params")
        return p

    def set_params(self, p):
        p = np.ascontiguousarray(p, np.float32)
        _check(load().dd_mlp_set_params(self.h, p.ctypes.data, p.size), "dd_mlp_set_params")

    def save(self, path):
        _check(load().dd_mlp_save(self.h, os.fsencode(path)), "dd_mlp_save")

    def load(self, path):
        _check(load().dd_mlp_load(self.h, os.fsencode(path)), "dd_mlp_load")

    @staticmethod
    def _dev(X):
        assert X.is_cuda and X.dtype.is_floating_point and X.is_contiguous()
        return X

    def forward(self, X):
        import torch
        X = self._dev(X)
        out = torch.empty((X.shape[0], 2), dtype=torch.float32, device=X.device)
        _check(load().dd_mlp_forward(self.h, X.data_ptr(), X.shape[0], out.data_ptr()), "dd_mlp_forward")
        return out

    def grad(self, X, u_star):
        """(gradient [DD_MLP_PARAMS], loss [1]) as CUDA tensors."""
        import torch
        X, u_star = self._dev(X), self._dev(u_star)
        g = torch.empty(DD_MLP_PARAMS, dtype=torch.float32, device=X.device)
        loss = torch.empty(1, dtype=torch.float32, device=X.device)
        _check(load().dd_mlp_grad(self.h, X.data_ptr(), u_star.data_ptr(), X.shape[0], g.data_ptr(),
                                  loss.data_ptr()), "dd_mlp_grad")
        return g, loss

    def train_step(self, X, u_star, lr, loss=None):
        """One Adam step; `loss` (CUDA tensor [1], optional) receives the loss."""
        X, u_star = self._dev(X), self._dev(u_star)
        _check(load().dd_mlp_train_step(self.h, X.data_ptr(), u_star.data_ptr(), X.shape[0], float(lr),
                                        loss.data_ptr() if loss is not None else None), "dd_mlp_train_step")


def dd_probe_peaks(stream_ptr=None):
    """(shared-memory atomic increments/s, L2 read bytes/s) measured on the device."""
    a, b = ctypes.c_double(), ctypes.c_double()
    _check(load().dd_probe_peaks(ctypes.byref(a), ctypes.byref(b), _VP(stream_ptr) if stream_ptr else None),
           "dd_probe_peaks")
    return a.value, b.value


def dd_stream_solve(h, stream, t_start, tau, hop, n_windows, params=(-1.0, 1.0, 1e-4, 0.0)):
    """Windows of a time-sorted stream (Events): (status, [results], ttc[k], first[k])."""
    n = int(n_windows)
    R = (dd_result * n)()
    ttc = np.zeros(n, np.float32)
    first = np.zeros(n, np.int64)
    p = window_params(params)
    rc = load().dd_stream_solve(h, ctypes.byref(stream.c), float(t_start), float(tau), float(hop), n, ctypes.byref(p),
                                R, ttc.ctypes.data, first.ctypes.data)
    res = [R[i].as_dict() for i in range(n)]
    if rc != DD_OK and all(r["status"] == DD_OK for r in res):
        raise DDError(rc, "dd_stream_solve")
    return rc, res, ttc, first


def dd_check_flags(reset=False):
    """(error word, checked build?) of the evaluation kernels' index tests."""
    f, c = ctypes.c_uint32(), ctypes.c_int32()
    _check(load().dd_check_flags(ctypes.byref(f), ctypes.byref(c), 1 if reset else 0), "dd_check_flags")
    return f.value, bool(c.value)


def dd_time_span(h, ev):
    """(t0, tau) of a batch measured from its earliest event (Sec. 3.3)."""
    a, b = ctypes.c_float(), ctypes.c_float()
    _check(load().dd_time_span(h, ctypes.byref(ev.c), ctypes.byref(a), ctypes.byref(b)), "dd_time_span")
    return a.value, b.value


LOG_KEYS = ("status", "D_star", "D_end", "contrast", "bound_gap", "K_hat", "gap_K", "nodes_expanded", "point_evals",
            "bound_evals", "event_warps", "cell_increments", "bound_increments", "rounds", "max_queue", "D_warm",
            "w_warm")


def write_pgm(path, img):
    """An image of counts as a binary PGM (16-bit, big-endian samples; counts
    above 65535 saturate), written from a host array; no graphics library."""
    a = np.asarray(img)
    if a.ndim != 2:
        raise ValueError("write_pgm takes one [H][W] image")
    a = np.minimum(a.astype(np.int64), 65535).astype(">u2")
    with open(path, "wb") as f:
        f.write(b"P5\n%d %d\n65535\n" % (a.shape[1], a.shape[0]))
        f.write(a.tobytes())


def read_pgm(path):
    """The counts of a PGM written by write_pgm."""
    with open(path, "rb") as f:
        data = f.read()
    parts = data.split(b"\n", 3)
    if parts[0] != b"P5":
        raise ValueError("not a binary PGM")
    W, H = (int(v) for v in parts[1].split())
    maxval = int(parts[2])
    dt = ">u2" if maxval > 255 else "u1"
    return np.frombuffer(parts[3], dtype=dt, count=W * H).reshape(H, W).astype(np.uint32)


def dd_resample_foe(W, H, foe_x, foe_y, W2, H2):
    a, b = ctypes.c_float(), ctypes.c_float()
    _check(load().dd_resample_foe(W, H, foe_x, foe_y, W2, H2, ctypes.byref(a), ctypes.byref(b)), "dd_resample_foe")
    return a.value, b.value


def dd_resample(h, ev, W, H, W2, H2, keep=0.25, seed=0):
    """The fast mode's window of events `ev` (W x H): torch CUDA tensors
    (x, y, t) of the kept events on the W2 x H2 frame."""
    import torch
    n = int(ev.c.n)
    x = torch.empty(max(n, 1), dtype=torch.int16, device="cuda")
    y = torch.empty(max(n, 1), dtype=torch.int16, device="cuda")
    t = torch.empty(max(n, 1), dtype=torch.float32, device="cuda")
    m = ctypes.c_int64()
    _check(load().dd_resample(h, ctypes.byref(ev.c), W, H, W2, H2, float(keep), int(seed), x.data_ptr(),
                              y.data_ptr(), t.data_ptr(), ctypes.byref(m)), "dd_resample")
    return x[:m.value], y[:m.value], t[:m.value]


def dd_contrast_noalloc(W, H, foe_x, foe_y, ev, D, stream_ptr=None):
    """Keys K[j] of dd_contrast without a context and without allocating
    device memory (events must be device tensors); see include/dd.h."""
    D = np.ascontiguousarray(D, dtype=np.float32)
    n = D.size
    K = (dd_i128 * max(n, 1))()
    _check(load().dd_contrast_noalloc(W, H, foe_x, foe_y, ctypes.byref(ev.c), D.ctypes.data, n,
                                      ctypes.cast(K, _VP), _VP(stream_ptr) if stream_ptr else None),
           "dd_contrast_noalloc")
    return [K[i].value() for i in range(n)]


class Server:
    """Continuous-batching server over a Context's geometry (dd_serve_*)."""

    def __init__(self, ctx, max_slots=0, max_events=1 << 20):
        h = _VP()
        _check(load().dd_serve_start(ctx.h, max_slots, max_events, ctypes.byref(h)), "dd_serve_start")
        self.h = h
        self._keep = {}
        s, e = ctypes.c_int32(), ctypes.c_int64()
        _check(load().dd_serve_slots(h, ctypes.byref(s), ctypes.byref(e)), "dd_serve_slots")
        self.slots, self.max_events = s.value, e.value

    @staticmethod
    def clock():
        return load().dd_serve_clock()

    def submit(self, ev, params=(-1.0, 1.0, 1e-4, 0.0), arrival=-1.0):
        t = ctypes.c_uint64()
        p = window_params(params)
        _check(load().dd_serve_submit(self.h, ctypes.byref(ev.c), ctypes.byref(p), float(arrival), ctypes.byref(t)),
               "dd_serve_submit")
        self._keep[t.value] = ev            # the arrays must outlive the request
        return t.value

    def _take(self, fn, ticket):
        r, lat = dd_result(), ctypes.c_double()
        rc = fn(self.h, ticket, ctypes.byref(r), ctypes.byref(lat))
        if rc == DD_PENDING:
            return None
        self._keep.pop(ticket, None)
        if rc != DD_OK:
            raise DDError(rc, "serve request %d" % ticket)
        d = r.as_dict()
        d["latency_s"] = lat.value
        return d

    def cancel(self, ticket):
        """Drop a waiting request or stop a running one after its current round;
        poll/wait then raise DDError with DD_ERR_CANCELLED."""
        _check(load().dd_serve_cancel(self.h, ticket), "dd_serve_cancel")

    def poll(self, ticket):
        return self._take(load().dd_serve_poll, ticket)

    def wait(self, ticket):
        return self._take(load().dd_serve_wait, ticket)

    def stats(self):
        a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(load().dd_serve_stats(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "dd_serve_stats")
        return {"rounds": a.value, "admitted": b.value, "peak_busy": c.value}

    def stop(self):
        if self.h:
            rc = load().dd_serve_stop(self.h)
            self.h = None
            self._keep.clear()
            _check(rc, "dd_serve_stop")


class Context:
    """A dd_ctx for one frame geometry (W x H, FOE)."""

    def __init__(self, W, H, foe_x, foe_y, pop_k=0, queue_capacity=0, band_rows=0, threads=0, max_rounds=0,
                 host_loop=0, max_splits=0, warp_to_start=0, polarity=0, fuse_span=0):
        self.W, self.H = int(W), int(H)
        self.planes = 2 if polarity else 1
        self.cfg = dd_config(pop_k, queue_capacity, band_rows, threads, max_rounds, host_loop, max_splits,
                             warp_to_start, polarity, fuse_span)
        self.h = dd_create(self.W, self.H, float(foe_x), float(foe_y), self.cfg)
        self._log = None

    @property
    def M(self):
        """Image cells of one hypothesis (both planes with polarity)."""
        return self.planes * self.W * self.H

    def set_log(self, path):
        """Append one JSON line per solved window to `path` (None: stop)."""
        if self._log:
            self._log.close()
        self._log = open(path, "a") if path else None

    def _logged(self, results, seconds, kind):
        if self._log:
            for r in results:
                rec = {k: r[k] for k in LOG_KEYS if k in r}
                rec.update(kind=kind, windows_in_call=len(results), call_us=seconds * 1e6)
                self._log.write(json.dumps(rec) + "\n")
            self._log.flush()
        return results

    def _image(self, img):
        shape = (-1, self.H, self.W) if self.planes == 1 else (-1, 2, self.H, self.W)
        return img.reshape(shape)

    @classmethod
    def tuned(cls, W, H, foe_x, foe_y, n_events, mode="single", **kw):
        """A context with the autotuned knobs for this geometry and size
        (autotune.py's table), falling back to the defaults."""
        from . import autotune
        knobs = autotune.lookup(W, H, n_events, mode) or {}
        knobs.update(kw)
        return cls(W, H, foe_x, foe_y, **knobs)

    def close(self):
        if self.h:
            dd_destroy(self.h)
            self.h = None
        if getattr(self, "_log", None):
            self._log.close()
            self._log = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_stream(self, stream_ptr):
        dd_set_stream(self.h, stream_ptr)

    def stats(self):
        return dd_get_stats(self.h)

    def reset_stats(self):
        dd_reset_stats(self.h)

    def set_timing(self, enable):
        dd_set_timing(self.h, enable)

    def launch_times(self):
        return dd_get_launch_times(self.h)

    def contrast(self, ev, D, want_iwe=False):
        K, S, N, img = dd_contrast(self.h, ev, D, want_iwe=want_iwe, M=self.M)
        return K, S, N, (self._image(img) if want_iwe else None)

    def bound(self, ev, D_lo, D_hi, want_iwe=False):
        K, S, N, img = dd_bound(self.h, ev, D_lo, D_hi, want_iwe=want_iwe, M=self.M)
        return K, S, N, (self._image(img) if want_iwe else None)

    def solve_batch(self, evs, params=None):
        """Solve several windows at once; params defaults to [-1, 1], 1e-4, 0."""
        if params is None:
            params = [(-1.0, 1.0, 1e-4, 0.0)] * len(evs)
        t0 = time.perf_counter()
        rc, res = dd_solve_batch(self.h, evs, params)
        self._logged(res, time.perf_counter() - t0, "batch")
        return rc, res

    def solve(self, ev, D_lo=-1.0, D_hi=1.0, tol_D=1e-4, gamma=0.0, trace_cap=0, warm=None):
        """One exact solve; warm = None, "model" or (D_warm, w_warm)."""
        t0 = time.perf_counter()
        if warm is not None:
            r = dd_solve_window(self.h, ev, (D_lo, D_hi, tol_D, gamma, warm), trace_cap)
        elif trace_cap:
            r = dd_solve_trace(self.h, ev, D_lo, D_hi, tol_D, gamma, trace_cap)
        else:
            r = dd_solve(self.h, ev, D_lo, D_hi, tol_D, gamma)
        self._logged([r], time.perf_counter() - t0, "single")
        return r

    def image(self, ev, D):
        """The image of warped events at D (Eq. 12): uint32 [H][W], or
        [2][H][W] with polarity planes."""
        return self.contrast(ev, np.array([D], np.float32), want_iwe=True)[3][0]

    def features(self, evs):
        return dd_features(self.h, evs)

    def resample(self, ev, W, H, keep=0.25, seed=0):
        """Events `ev` of a W x H window in this context's (coarser) frame:
        the fast mode's pre-pass (dd_resample); returns Events on the device."""
        x, y, t = dd_resample(self.h, ev, W, H, self.W, self.H, keep, seed)
        return Events(x.contiguous(), y.contiguous(), t.contiguous(), ev.c.t0, ev.c.tau)

    def time_span(self, ev):
        """(t0, tau) of a batch measured from its earliest event (Sec. 3.3)."""
        return dd_time_span(self.h, ev)

    def stream_solve(self, stream, t_start, tau, hop, n_windows, params=(-1.0, 1.0, 1e-4, 0.0)):
        """The stream-wise estimation (dd_stream_solve): windows of `stream`."""
        return dd_stream_solve(self.h, stream, t_start, tau, hop, n_windows, params)

    def set_warm_model(self, mlp):
        """The model DD_WARM_MODEL windows start from (None clears); keep it alive."""
        _check(load().dd_set_warm_model(self.h, mlp.h if mlp is not None else None), "dd_set_warm_model")
        self._model = mlp
