"""Learned surrogate of the sweep, for parameter screening.

A small BF16 MLP ensemble maps (ln n_b/n_p, ln gamma_b, k_p L, k_p xi,
omega_p t, |k_perp|, k_perp angle) to the log growth envelope and the
dominant mode class (CFI / OTSI).  The solver generates the training data
(qs_sur_points on recorded snapshots), the library's own kernels train the
network (qs_mlp_train_step) and answer queries (qs_mlp_infer); queries the
ensemble is unsure about (variance above a threshold) are flagged and
answered by the solver instead.

This module only sequences C-ABI calls and moves buffers; every arithmetic
step runs in libqs.so.
"""
from __future__ import annotations

import ctypes
import time

import numpy as np

from . import lib, QSError, Solver, REC_MAG, Allocator, Params, make_params

_vp = ctypes.c_void_p
_fp = ctypes.POINTER(ctypes.c_float)


def _setup():
    L = lib
    i64 = ctypes.c_int64
    L.qs_mlp_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                ctypes.c_int, ctypes.c_uint64, ctypes.POINTER(Allocator), _vp,
                                ctypes.POINTER(_vp)]
    L.qs_mlp_set_norm.argtypes = [_vp, _vp, i64, _vp]
    L.qs_mlp_params.argtypes = [_vp, ctypes.c_int, _fp, i64, ctypes.c_int]
    L.qs_mlp_layout.argtypes = [_vp, ctypes.POINTER(i64), ctypes.POINTER(i64), _fp]
    L.qs_mlp_train_step.argtypes = [_vp, _vp, _vp, i64, ctypes.c_float, ctypes.c_int, _fp]
    L.qs_mlp_grads.argtypes = [_vp, ctypes.c_int, _fp, i64]
    L.qs_mlp_infer.argtypes = [_vp, _vp, i64, _vp, _vp, _vp, ctypes.c_float]
    L.qs_mlp_last_error.argtypes = [_vp]
    L.qs_mlp_last_error.restype = ctypes.c_char_p
    L.qs_mlp_free.argtypes = [_vp]
    L.qs_mlp_free.restype = None
    L.qs_sur_points.argtypes = [_vp, _vp, ctypes.c_size_t, ctypes.c_double, i64, ctypes.c_uint64, _vp, _vp]
    L.qs_sur_train.argtypes = [_vp, _vp, _vp, i64, ctypes.c_char_p, ctypes.POINTER(_vp)]
    L.qs_sur_infer.argtypes = [_vp, _vp, i64, _vp, _vp, _vp]
    L.qs_sur_losses.argtypes = [_vp, _fp, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    L.qs_sur_set_threshold.argtypes = [_vp, ctypes.c_float]
    L.qs_sur_free.argtypes = [_vp]
    L.qs_sur_free.restype = None
    L.qs_sur_screen.argtypes = [_vp, _vp, ctypes.POINTER(Params), ctypes.c_int, ctypes.c_uint64, ctypes.c_double,
                                _vp, i64, _vp, _vp, _vp, ctypes.POINTER(i64)]
    L.qs_sur_screen.restype = ctypes.c_int
    for n in ("qs_mlp_create", "qs_mlp_set_norm", "qs_mlp_params", "qs_mlp_layout", "qs_mlp_train_step",
              "qs_mlp_grads", "qs_mlp_infer", "qs_sur_points", "qs_sur_train", "qs_sur_infer", "qs_sur_losses",
              "qs_sur_set_threshold"):
        getattr(L, n).restype = ctypes.c_int


_setup()


def _ptr(t):
    return _vp(t.data_ptr())


class MLP:
    """Ensemble of BF16 MLPs n_in -> width^depth (GELU) -> 2."""

    def __init__(self, n_in=7, width=256, depth=3, ensemble=4, max_batch=16384, seed=0, stream=None):
        import torch
        self.torch = torch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = _vp()
        st = lib.qs_mlp_create(n_in, width, depth, 2, ensemble, max_batch, seed, None,
                               _vp(self.stream.cuda_stream), ctypes.byref(h))
        if st != 0:
            raise QSError(st, "qs_mlp_create failed")
        self.h = h
        self.n_in, self.width, self.depth, self.E, self.max_batch = n_in, width, depth, ensemble, max_batch
        n = ctypes.c_int64()
        offs = (ctypes.c_int64 * (2 * (depth + 1)))()
        lib.qs_mlp_layout(self.h, ctypes.byref(n), offs, None)
        self.nparam = n.value
        self.offsets = list(offs)

    def _chk(self, st):
        if st != 0:
            raise QSError(st, lib.qs_mlp_last_error(self.h).decode())

    def close(self):
        if getattr(self, "h", None):
            lib.qs_mlp_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_norm(self, X, Y=None):
        self._chk(lib.qs_mlp_set_norm(self.h, _ptr(X), X.shape[0], _ptr(Y) if Y is not None else None))

    def norm(self):
        n = ctypes.c_int64()
        buf = (ctypes.c_float * 64)()
        self._chk(lib.qs_mlp_layout(self.h, ctypes.byref(n), None, buf))
        a = np.array(buf[:], dtype=np.float64)
        return a[:32], a[32:], float(a[62]), float(a[63])

    def params(self, member=0):
        out = np.zeros(self.nparam, np.float32)
        self._chk(lib.qs_mlp_params(self.h, member, out.ctypes.data_as(_fp), self.nparam, 0))
        return out

    def set_params(self, flat, member=0):
        a = np.ascontiguousarray(flat, np.float32)
        self._chk(lib.qs_mlp_params(self.h, member, a.ctypes.data_as(_fp), self.nparam, 1))

    def grads(self, member=0):
        out = np.zeros(self.nparam, np.float32)
        self._chk(lib.qs_mlp_grads(self.h, member, out.ctypes.data_as(_fp), self.nparam))
        return out

    def layers(self, flat):
        """Split a flat parameter vector into [(W [out][in], b [out])]."""
        res = []
        ins = [(self.n_in + 15) // 16 * 16] + [self.width] * self.depth
        outs = [self.width] * self.depth + [2]
        for l in range(self.depth + 1):
            w0, b0 = self.offsets[2 * l], self.offsets[2 * l + 1]
            W = flat[w0:w0 + ins[l] * outs[l]].reshape(outs[l], ins[l])
            b = flat[b0:b0 + outs[l]]
            res.append((W, b))
        return res

    def train_step(self, X, Y, lr, update=True, want_loss=False):
        loss = ctypes.c_float()
        self._chk(lib.qs_mlp_train_step(self.h, _ptr(X), _ptr(Y), X.shape[0], float(lr), 1 if update else 0,
                                        ctypes.byref(loss) if want_loss else None))
        return loss.value if want_loss else None

    def infer(self, X, var_threshold=float("inf")):
        torch = self.torch
        n = X.shape[0]
        mean = torch.empty((n, 2), dtype=torch.float32, device=X.device)
        var = torch.empty_like(mean)
        mask = torch.empty(n, dtype=torch.uint8, device=X.device)
        self._chk(lib.qs_mlp_infer(self.h, _ptr(X), n, _ptr(mean), _ptr(var), _ptr(mask),
                                   float(min(var_threshold, 3e38))))
        return mean, var, mask


class SurModel:
    """A surrogate trained in one library call (qs_sur_train): the whole
    training loop, shuffles included, runs behind the C ABI."""

    def __init__(self, X, Y, solver=None, **cfg):
        import json
        self.h = _vp()
        js = json.dumps({k: float(v) for k, v in cfg.items()}).encode()
        st = lib.qs_sur_train(solver.ctx if solver is not None else None, _ptr(X), _ptr(Y), X.shape[0], js,
                              ctypes.byref(self.h))
        if st != 0:
            raise QSError(st, "qs_sur_train failed")

    def losses(self):
        n = ctypes.c_int()
        lib.qs_sur_losses(self.h, None, 0, ctypes.byref(n))
        out = (ctypes.c_float * max(n.value, 1))()
        lib.qs_sur_losses(self.h, out, n.value, ctypes.byref(n))
        return list(out)[:n.value]

    def set_threshold(self, thr):
        lib.qs_sur_set_threshold(self.h, float(min(thr, 3e38)))

    def infer(self, X):
        import torch
        n = X.shape[0]
        mean = torch.empty((n, 2), dtype=torch.float32, device=X.device)
        var = torch.empty_like(mean)
        mask = torch.empty(n, dtype=torch.uint8, device=X.device)
        st = lib.qs_sur_infer(self.h, _ptr(X), n, _ptr(mean), _ptr(var), _ptr(mask))
        if st != 0:
            raise QSError(st, "qs_sur_infer failed")
        return mean, var, mask

    def screen(self, problems, X, noise_seed, amplitude=1e-6, prec="fp32", lend=None):
        """Screening with the solver as fallback (qs_sur_screen): the ensemble
        answers every query of X; queries above the variance threshold are
        answered by solver runs of their parameter sets (`problems`, the sets
        the queries may name).  Returns (y, var, mask, n_solved): mask = 1
        where the solver answered (y[:, 1] is then a saturated logit)."""
        import torch
        n = X.shape[0]
        keep = []
        arr = (Params * len(problems))(*[make_params(q, prec, keep) for q in problems])
        y = torch.empty((n, 2), dtype=torch.float32, device=X.device)
        var = torch.empty_like(y)
        mask = torch.empty(n, dtype=torch.uint8, device=X.device)
        ns = ctypes.c_int64()
        st = lib.qs_sur_screen(self.h, lend.ctx if lend is not None else None, arr, len(problems),
                               int(noise_seed) & 0xFFFFFFFFFFFFFFFF, float(amplitude), _ptr(X), n, _ptr(y),
                               _ptr(var), _ptr(mask), ctypes.byref(ns))
        if st != 0:
            raise QSError(st, lib.qs_last_error(lend.ctx if lend is not None else None).decode())
        return y, var, mask, ns.value

    def close(self):
        if self.h:
            lib.qs_sur_free(self.h)
            self.h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def generate(problems, snapshot_steps, n_per_snapshot, seed=0, amplitude=1e-6, prec="fp32",
             noise_seed=0, stream=None):
    """Run the solver over `problems` (one context, instances batched) and
    draw n_per_snapshot samples at each requested slow-time step.
    Returns device tensors X [n][7], Y [n][2] and the solver seconds."""
    import torch
    s = Solver(problems, prec=prec, stream=stream)
    s.seed_noise(noise_seed, amplitude)
    n_tot = n_per_snapshot * len(snapshot_steps)
    X = torch.empty((n_tot, 7), dtype=torch.float32, device="cuda")
    Y = torch.empty((n_tot, 2), dtype=torch.float32, device="cuda")
    t0 = time.perf_counter()
    for k, stp in enumerate(sorted(snapshot_steps)):
        d = stp - s.step_count
        if d > 0:
            s.step(d)
        snap = s.diag(REC_MAG, host=False)
        st = lib.qs_sur_points(s.ctx, _ptr(snap), snap.numel() * 8, float(amplitude), n_per_snapshot,
                               (seed * 1000003 + k) & 0xFFFFFFFFFFFFFFFF,
                               _ptr(X[k * n_per_snapshot:]), _ptr(Y[k * n_per_snapshot:]))
        if st != 0:
            raise QSError(st, lib.qs_last_error(s.ctx).decode())
        del snap
    s.sync()
    secs = time.perf_counter() - t0
    s.close()
    return X, Y, secs


def train(X, Y, epochs=20, batch=8192, lr=1e-3, ensemble=4, width=256, depth=3, seed=0, log=None):
    """Train an ensemble on device tensors X, Y; returns the MLP and the
    per-epoch mean losses."""
    import torch
    m = MLP(width=width, depth=depth, ensemble=ensemble, max_batch=batch, seed=seed)
    m.set_norm(X, Y)
    n = X.shape[0]
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    losses = []
    for ep in range(epochs):
        perm = torch.randperm(n, device="cuda", generator=g)
        Xs, Ys = X[perm].contiguous(), Y[perm].contiguous()
        tot, cnt = 0.0, 0
        lr_ep = lr * 0.5 * (1 + np.cos(np.pi * ep / epochs))
        for b0 in range(0, n - batch + 1, batch):
            l = m.train_step(Xs[b0:b0 + batch], Ys[b0:b0 + batch], lr_ep, want_loss=(b0 == 0))
            if b0 == 0:
                tot += l
                cnt += 1
        losses.append(tot / max(cnt, 1))
        if log:
            log(f"epoch {ep} loss {losses[-1]:.4f}")
    return m, losses


def score(mean, Y):
    """Envelope RMSE / MAE and class accuracy of outputs `mean` [n][2] (target
    units, class logit) against labels Y [n][2]."""
    yt = Y[:, 0]
    err = (mean[:, 0] - yt)
    cls = (mean[:, 1] > 0).float()
    return {
        "rmse": float(err.pow(2).mean().sqrt()),
        "mae": float(err.abs().mean()),
        "target_std": float(yt.std()),
        "accuracy": float((cls == Y[:, 1]).float().mean()),
    }


def evaluate(m, X, Y):
    """Held-out errors of the ensemble alone (no fallback)."""
    mean, _, _ = m.infer(X)
    return score(mean, Y)
