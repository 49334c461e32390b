"""Finite-width beam on a periodic transverse grid (qs_r2_* of libqs.so).

Thin ctypes wrapper: argument marshalling only; the plasma march, the FFT
screened-Poisson solve and the push run in the library's kernels.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import lib, QSError, Species

_vp = ctypes.c_void_p


class R2Params(ctypes.Structure):
    _fields_ = [("species", Species), ("gamma_b", ctypes.c_double), ("n_xi", ctypes.c_int),
                ("dxi", ctypes.c_double), ("dt", ctypes.c_double), ("n_perp", ctypes.c_int),
                ("L_perp", ctypes.c_double), ("sigma_r", ctypes.c_double), ("uniform", ctypes.c_int)]


lib.qs_r2_init.argtypes = [ctypes.POINTER(R2Params), _vp, _vp, ctypes.POINTER(_vp)]
lib.qs_r2_seed.argtypes = [_vp, ctypes.c_uint64, ctypes.c_double, ctypes.c_double, _vp, ctypes.c_size_t,
                           ctypes.c_int]
lib.qs_r2_step.argtypes = [_vp, ctypes.c_int]
lib.qs_r2_read.argtypes = [_vp, ctypes.c_int, _vp, ctypes.c_size_t, ctypes.c_int]
lib.qs_r2_sync.argtypes = [_vp]
lib.qs_r2_launch_count.argtypes = [_vp]
lib.qs_r2_launch_count.restype = ctypes.c_int64
lib.qs_r2_free.argtypes = [_vp]
lib.qs_r2_free.restype = None
for _n in ("qs_r2_init", "qs_r2_seed", "qs_r2_step", "qs_r2_read", "qs_r2_sync"):
    getattr(lib, _n).restype = ctypes.c_int


class RealSpace:
    def __init__(self, problem: dict, stream=None):
        import torch
        assert problem["ny"] == problem["nz"] and problem["Ly"] == problem["Lz"]
        q, m, d = problem["species"][0]
        p = R2Params(Species(q, m, d), float(problem["gamma_b"]), int(problem["n_xi"]), float(problem["dxi"]),
                     float(problem["dt"]), int(problem["ny"]), float(problem["Ly"]),
                     float(problem.get("sigma_r", 1.0)), 1 if problem.get("transverse") == "uniform" else 0)
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = _vp()
        st = lib.qs_r2_init(ctypes.byref(p), None, _vp(self.stream.cuda_stream), ctypes.byref(h))
        if st != 0:
            raise QSError(st, "qs_r2_init failed")
        self.h = h
        self.shape = (int(problem["n_xi"]), int(problem["ny"]), int(problem["nz"]))

    def seed(self, seed=0, amplitude=1e-6, offset=0.0, noise=None):
        if noise is None:
            st = lib.qs_r2_seed(self.h, int(seed), float(amplitude), float(offset), None, 0, 1)
        elif isinstance(noise, np.ndarray):
            a = np.ascontiguousarray(noise, np.float32)
            st = lib.qs_r2_seed(self.h, 0, float(amplitude), float(offset), a.ctypes.data_as(_vp), a.nbytes, 1)
        else:
            t = noise.contiguous()
            st = lib.qs_r2_seed(self.h, 0, float(amplitude), float(offset), _vp(t.data_ptr()),
                                t.numel() * 4, 0)
        if st != 0:
            raise QSError(st, "qs_r2_seed failed")

    def step(self, n=1):
        st = lib.qs_r2_step(self.h, int(n))
        if st != 0:
            raise QSError(st, "qs_r2_step failed")

    def sync(self):
        st = lib.qs_r2_sync(self.h)
        if st != 0:
            raise QSError(st, "device error in the real-space sweep")

    def read(self, what=0):
        out = np.empty(self.shape, np.float32)
        st = lib.qs_r2_read(self.h, int(what), out.ctypes.data_as(_vp), out.nbytes, 1)
        if st != 0:
            raise QSError(st, "qs_r2_read failed")
        return out

    def launch_count(self):
        return int(lib.qs_r2_launch_count(self.h))

    def close(self):
        if getattr(self, "h", None):
            lib.qs_r2_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
