"""Synthetic windows generated on the GPU (synth/gen.cu), for workloads too
large to generate with numpy in reasonable time.  Same windows as
synth.descent.make_window (event order aside); tests/test_synth_gpu.py
checks that."""
import ctypes
import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.cu")
_LIB = os.path.join(_HERE, "libsynth.so")
_lib = None


def build(force=False):
    """Compile gen.cu into libsynth.so (binary64 without FMA contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    nvcc = "nvcc" if subprocess.run(["which", "nvcc"], capture_output=True).returncode == 0 else "/usr/local/cuda/bin/nvcc"
    tmp = _LIB + ".%d.tmp" % os.getpid()
    subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-fmad=false", "-shared",
                           "-Xcompiler", "-fPIC,-ffp-contract=off", "-o", tmp, _SRC])
    os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.synth_window_gpu.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
        L.synth_window_gpu.restype = ctypes.c_int
        _lib = L
    return _lib


class GpuWindow:
    """A window whose SoA events live in torch CUDA tensors."""

    def __init__(self, spec, x, y, t, p=None):
        (self.W, self.H, self.foe_x, self.foe_y, self.n_signal, self.n_points, self.n_noise, self.D_true,
         tau, self.seed) = spec
        import numpy as np
        self.tau = float(np.float32(tau))
        self.t0 = 0.0
        self.x, self.y, self.t, self.p = x, y, t, p

    @property
    def n(self):
        return int(self.x.shape[0])


def make_window_gpu(spec, device="cuda", stream=None, polarity=False):
    """Generate make_window(*spec) on the GPU; returns a GpuWindow (with
    its int8 polarities in .p when polarity=True, else .p = None)."""
    import torch
    W, H, fx, fy, n_sig, n_pts, n_noise, D, tau, seed = spec
    n = int(n_sig) + int(n_noise)
    x = torch.empty(n, dtype=torch.int16, device=device)
    y = torch.empty(n, dtype=torch.int16, device=device)
    t = torch.empty(n, dtype=torch.float32, device=device)
    p = torch.empty(n, dtype=torch.int8, device=device) if polarity else None
    s = stream if stream is not None else torch.cuda.current_stream().cuda_stream
    rc = lib().synth_window_gpu(int(W), int(H), float(fx), float(fy), int(n_sig), int(n_pts), int(n_noise), float(D),
                                float(tau), int(seed), x.data_ptr(), y.data_ptr(), t.data_ptr(),
                                p.data_ptr() if polarity else None, s)
    if rc != 0:
        raise RuntimeError("synth_window_gpu failed (%d)" % rc)
    return GpuWindow(spec, x, y, t, p)


def make_stream_gpu(stream, k0, k1, n_scale=1.0):
    """The continuous descent stream (slots k0..k1-1 of synth.descent.
    stream_slot_spec5) generated on the GPU: torch CUDA tensors (x, y, t)
    sorted by time; times shifted as make_window(t0=...) shifts them
    (binary64 sum rounded to binary32)."""
    import torch
    from .descent import stream_slot_spec5
    xs, ys, ts = [], [], []
    for k in range(k0, k1):
        spec, tk = stream_slot_spec5(stream, k, n_scale)
        w = make_window_gpu(spec)
        xs.append(w.x)
        ys.append(w.y)
        ts.append((w.t.double() + tk).float())
    x, y, t = torch.cat(xs), torch.cat(ys), torch.cat(ts)
    t, o = torch.sort(t, stable=True)
    return x[o].contiguous(), y[o].contiguous(), t.contiguous()
