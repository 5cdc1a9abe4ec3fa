"""Device-side generation of the synthetic samples (same draws as synth.workload, on the GPU).

Used for workloads too large to draw on the host (the 16384-parameter, 10^6-sample step).
"""
import ctypes
import os

import numpy as np

from .workload import make_model

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libblmsynth.so")
_lib = None


def _load():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libblmsynth.so is not built (synth.device_build.build())")
        _lib = ctypes.CDLL(LIB_PATH)
        _lib.blmsynth_samples.restype = ctypes.c_int
        _lib.blmsynth_samples.argtypes = [ctypes.c_int64, ctypes.c_int64, ctypes.c_int64,
                                          ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                                          ctypes.c_double] + [ctypes.c_void_p] * 7 + \
                                         [ctypes.c_int, ctypes.c_int64, ctypes.c_void_p]
    return _lib


class DeviceModel:
    def __init__(self, wl, device="cuda:0"):
        import torch
        self.wl = wl
        m = make_model(wl)
        self.u = torch.from_numpy(np.ascontiguousarray(m.u)).to(device)
        self.sigma = torch.from_numpy(m.sigma).to(device)
        self.g = torch.from_numpy(m.g).to(device)
        self.mu = torch.from_numpy(m.mu).to(device)


def fill(dm, s0, O, G, E, stream=0):
    """Write samples s0 .. s0 + O.shape[0] - 1 into the device tensors O, G (rows x ld) and E."""
    import torch
    wl = dm.wl
    lib = _load()
    f32 = 1 if O.dtype == torch.float32 else 0
    rc = lib.blmsynth_samples(wl.n, int(s0), int(O.shape[0]), wl.seed, wl.opt,
                              0 if wl.noise == "normal" else 1, float(wl.offset),
                              dm.u.data_ptr(), dm.sigma.data_ptr(), dm.g.data_ptr(),
                              dm.mu.data_ptr(), O.data_ptr(), G.data_ptr(), E.data_ptr(), f32,
                              int(O.stride(0)), ctypes.c_void_p(int(stream)))
    if rc != 0:
        raise RuntimeError("blmsynth_samples failed with CUDA error %d" % rc)
