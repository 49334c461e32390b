"""B300-native linearised quasistatic (QSA) beam-plasma sweep.

Thin ctypes binding over ``libqs.so`` (include/qs.h).  The binding only
marshals arguments: every step of the sweep runs in the library's sm_103a
kernels.  PyTorch supplies device memory (its caching allocator, through the
library's allocator callback) and the CUDA stream.  There is no CPU or
fallback path: if the library cannot be loaded the import fails.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# QS_LIBRARY selects another build of the library (the bounds-checked
# libqs_checked.so); the default is the ordinary build in this directory
LIB_PATH = os.environ.get("QS_LIBRARY") or os.path.join(_HERE, "libqs.so")

# --- enums (qs.h) ------------------------------------------------------------
QS_OK, QS_ERR_ARG, QS_ERR_OOM, QS_ERR_CUDA, QS_ERR_TIMEOUT, QS_ERR_NONFINITE, QS_ERR_STATE, \
    QS_ERR_UNSUPPORTED, QS_ERR_BOUNDS = range(9)
BUILD_CHECK_BOUNDS = 1
GEOM = {"klist": 0, "kgrid2": 1, "real2": 2}
PREC = {"fp64": 0, "fp32": 1}
MODEL = {"full": 0, "reduced": 1}
FRONT = {"quiescent": 0, "equilibrium": 1, "held": 2}
PROFILE = {"flattop": 0, "gaussian": 1, "ramp_flattop": 2, "user": 3}
SEED_NOISE, SEED_IMPULSE, SEED_USER, SEED_STATE = range(4)
REC_MAG, REC_NP, REC_MODEMAX = 1, 2, 4
DIAG_XIMAX, DIAG_STATE, DIAG_WAKE0 = 8, 16, 32
Q_N_MODES, Q_MODES_PADDED, Q_N_INST, Q_TOTAL_CELLS, Q_STEP, Q_STATE_BYTES, Q_SNAPSHOT_BYTES, \
    Q_CELL_OFFSET, Q_LAUNCH, Q_RES_EVERY = range(10)

EXPORTS = ["qs_init", "qs_seed", "qs_step", "qs_record", "qs_diag", "qs_query", "qs_modes",
           "qs_set_launch", "qs_get_launch", "qs_tune", "qs_step_graph", "qs_step_green", "qs_sync",
           "qs_launch_count", "qs_last_error", "qs_free"]


class QSError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"qs status {status}: {msg}")
        self.status = status


class Species(ctypes.Structure):
    _fields_ = [("q", ctypes.c_double), ("m", ctypes.c_double), ("density_ratio", ctypes.c_double)]


class Params(ctypes.Structure):
    _fields_ = [
        ("geom", ctypes.c_int), ("prec", ctypes.c_int), ("model", ctypes.c_int),
        ("front", ctypes.c_int), ("n_species", ctypes.c_int), ("species", Species * 2),
        ("gamma_b", ctypes.c_double), ("profile", ctypes.c_int),
        ("length", ctypes.c_double), ("sigma_xi", ctypes.c_double), ("center_xi", ctypes.c_double),
        ("ramp_len", ctypes.c_double), ("user_profile", ctypes.POINTER(ctypes.c_double)),
        ("n_xi", ctypes.c_int), ("dxi", ctypes.c_double), ("dt", ctypes.c_double),
        ("n_k", ctypes.c_int), ("k_list", ctypes.POINTER(ctypes.c_double)),
        ("nkx", ctypes.c_int), ("nky", ctypes.c_int), ("kmax", ctypes.c_double),
        ("disc_mask", ctypes.c_int), ("held_front", ctypes.POINTER(ctypes.c_double)),
    ]


class Allocator(ctypes.Structure):
    _fields_ = [("alloc", ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)),
                ("free", ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)),
                ("user", ctypes.c_void_p)]


class Launch(ctypes.Structure):
    _fields_ = [("warps_per_cta", ctypes.c_int), ("prefetch", ctypes.c_int),
                ("persistent", ctypes.c_int), ("ctas_per_sm", ctypes.c_int), ("variant", ctypes.c_int),
                ("scan_cells", ctypes.c_int)]


def _source_hash():
    """The build script's hash of the library sources (loaded by path: the
    build script imports nothing from this package)."""
    import importlib.util
    spec = importlib.util.spec_from_file_location("qs_build_hash", os.path.join(_HERE, "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod.source_hash()


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with "
                          f"`python paper_2607_24234_b300/build.py` (nvcc, sm_103a)")
    try:
        built = open(LIB_PATH + ".srchash").read().strip()
    except OSError:
        built = None
    if built != _source_hash():
        raise ImportError(f"{LIB_PATH} was not built from the current sources: rebuild it with "
                          f"`python paper_2607_24234_b300/build.py`")
    L = ctypes.CDLL(LIB_PATH)
    vp, i64 = ctypes.c_void_p, ctypes.c_int64
    L.qs_init.argtypes = [ctypes.POINTER(Params), ctypes.c_int, ctypes.POINTER(Params),
                          ctypes.POINTER(Allocator), vp, ctypes.POINTER(vp)]
    L.qs_seed.argtypes = [vp, ctypes.c_uint64, ctypes.c_double, ctypes.c_int, vp, ctypes.c_size_t,
                          ctypes.c_int]
    L.qs_step.argtypes = [vp, ctypes.c_int]
    L.qs_record.argtypes = [vp, ctypes.c_int, ctypes.c_int, vp, ctypes.c_size_t]
    L.qs_diag.argtypes = [vp, ctypes.c_int, vp, ctypes.c_size_t, ctypes.c_int]
    L.qs_query.argtypes = [vp, ctypes.c_int, i64, ctypes.POINTER(i64)]
    L.qs_modes.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    L.qs_set_launch.argtypes = [vp, ctypes.POINTER(Launch)]
    L.qs_get_launch.argtypes = [vp, ctypes.POINTER(Launch)]
    L.qs_tune.argtypes = [vp, ctypes.c_int, ctypes.c_char_p]
    L.qs_step_graph.argtypes = [vp, ctypes.c_int]
    L.qs_step_green.argtypes = [vp, ctypes.c_int]
    L.qs_sync.argtypes = [vp]
    L.qs_debug_waits.argtypes = [vp, i64, ctypes.c_int]
    L.qs_debug_waits.restype = ctypes.c_int
    L.qs_debug_bounds.argtypes = [vp, i64]
    L.qs_debug_bounds.restype = ctypes.c_int
    L.qs_debug_canary.argtypes = [vp, ctypes.c_int]
    L.qs_debug_canary.restype = ctypes.c_int
    L.qs_build_flags.argtypes = []
    L.qs_build_flags.restype = ctypes.c_int
    L.qs_launch_count.argtypes = [vp]
    L.qs_launch_count.restype = i64
    L.qs_last_error.argtypes = [vp]
    L.qs_last_error.restype = ctypes.c_char_p
    L.qs_free.argtypes = [vp]
    L.qs_free.restype = None
    L.qs_sweep_noalloc.argtypes = [ctypes.POINTER(Params), vp, vp, ctypes.POINTER(ctypes.c_int), i64,
                                   ctypes.c_int, ctypes.POINTER(ctypes.c_int), vp]
    L.qs_sweep_noalloc.restype = ctypes.c_int
    L.qs_probe_alu.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, i64, vp, vp,
                               ctypes.POINTER(ctypes.c_double)]
    L.qs_probe_alu.restype = ctypes.c_int
    L.qs_growth_bound.argtypes = [ctypes.POINTER(Params), ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]
    L.qs_growth_bound.restype = ctypes.c_int
    for name in ("qs_init", "qs_seed", "qs_step", "qs_record", "qs_diag", "qs_query", "qs_modes",
                 "qs_set_launch", "qs_get_launch", "qs_tune", "qs_step_graph", "qs_step_green", "qs_sync"):
        getattr(L, name).restype = ctypes.c_int
    return L


lib = _load()


PROBE_FFMA2, PROBE_FFMA, PROBE_DFMA, PROBE_DADD, PROBE_DMUL = range(5)


def probe_alu(kind: int, blocks: int, threads: int, iters: int, sink, stream) -> float:
    """Enqueue one arithmetic-rate probe launch (qs_probe_alu) on `stream`;
    returns the FMA lane-operations it performs.  `sink`: a device tensor of
    at least 8 bytes."""
    ops = ctypes.c_double()
    st = lib.qs_probe_alu(int(kind), int(blocks), int(threads), int(iters), ctypes.c_void_p(sink.data_ptr()),
                          ctypes.c_void_p(stream.cuda_stream), ctypes.byref(ops))
    if st != QS_OK:
        raise QSError(st, "qs_probe_alu")
    return ops.value


def growth_bound(problem: dict, prec: str = "fp32"):
    """(e-folds per step bound, resident renormalisation interval) of a
    problem (qs_growth_bound; host only)."""
    keep = []
    prm = make_params(problem, prec, keep)
    g, ev = ctypes.c_double(), ctypes.c_int()
    st = lib.qs_growth_bound(ctypes.byref(prm), ctypes.byref(g), ctypes.byref(ev))
    if st != QS_OK:
        raise QSError(st, lib.qs_last_error(None).decode())
    return g.value, ev.value


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def make_params(problem: dict, prec: str, keep: list, held=None) -> Params:
    """qs_params from a problem dict (see synth); `keep` holds arrays alive."""
    p = Params()
    p.geom = GEOM[problem.get("geom", "klist")]
    p.prec = PREC[prec]
    p.model = MODEL[problem.get("model", "full")]
    p.front = FRONT[problem.get("front", "quiescent")]
    sp = problem["species"]
    p.n_species = len(sp)
    for i, (q, m, d) in enumerate(sp):
        p.species[i] = Species(float(q), float(m), float(d))
    p.gamma_b = float(problem["gamma_b"])
    p.profile = PROFILE[problem.get("profile", "flattop")]
    p.n_xi = int(problem["n_xi"])
    p.dxi = float(problem["dxi"])
    p.dt = float(problem["dt"])
    p.length = float(problem.get("length", p.n_xi * p.dxi))
    p.sigma_xi = float(problem.get("sigma_xi", 1.0))
    p.center_xi = float(problem.get("center_xi", 0.0))
    p.ramp_len = float(problem.get("ramp_len", 0.0))
    if p.profile == PROFILE["user"]:
        up = np.ascontiguousarray(problem["user_profile"], np.float64)
        keep.append(up)
        p.user_profile = _dptr(up)
    if p.geom == GEOM["klist"]:
        k = np.ascontiguousarray(problem["k_list"], np.float64)
        keep.append(k)
        p.n_k = len(k)
        p.k_list = _dptr(k)
    else:
        p.nkx, p.nky = int(problem["nkx"]), int(problem["nky"])
        p.kmax = float(problem["kmax"])
        p.disc_mask = int(problem.get("disc_mask", 1))
    if held is not None:
        h = np.ascontiguousarray(held, np.float64)
        keep.append(h)
        p.held_front = _dptr(h)
    return p


class Solver:
    """One context: n_inst instances of a problem (or a list of per-instance
    problems sharing the k set), advanced together on one CUDA stream."""

    def __init__(self, problem, prec: str = "fp32", stream=None, torch_alloc: bool = True,
                 held=None):
        import torch
        self.torch = torch
        self._keep = []
        probs = problem if isinstance(problem, (list, tuple)) else [problem]
        self.problems = list(probs)
        self.prec = prec
        base = make_params(probs[0], prec, self._keep, held=held)
        per = None
        if len(probs) > 1:
            per = (Params * len(probs))(*[make_params(q, prec, self._keep, held=held) for q in probs])
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._alloc = None
        if torch_alloc:
            dev = torch.cuda.current_device()
            stream_ = self.stream

            def _a(n, u):
                try:
                    return torch.cuda.caching_allocator_alloc(int(n), dev, stream_)
                except Exception:
                    return None

            def _f(ptr, u):
                torch.cuda.caching_allocator_delete(ptr)

            self._alloc = Allocator(Allocator._fields_[0][1](_a), Allocator._fields_[1][1](_f), None)
        ctx = ctypes.c_void_p()
        st = lib.qs_init(ctypes.byref(base), len(probs), per,
                         ctypes.byref(self._alloc) if self._alloc else None,
                         ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(ctx))
        if st != QS_OK:
            raise QSError(st, lib.qs_last_error(None).decode())
        self.ctx = ctx
        self.n_modes = self.query(Q_N_MODES)
        self.Mp = self.query(Q_MODES_PADDED)
        self.n_inst = self.query(Q_N_INST)
        self.cells = self.query(Q_TOTAL_CELLS)
        self.cell_off = [self.query(Q_CELL_OFFSET, i) for i in range(self.n_inst)]
        self.n_xi = [int(q["n_xi"]) for q in probs] if len(probs) > 1 else [int(probs[0]["n_xi"])]
        self._rec = None

    # -- plumbing ---------------------------------------------------------------
    def _chk(self, st):
        if st != QS_OK:
            raise QSError(st, lib.qs_last_error(self.ctx).decode())

    def query(self, what, arg=0):
        v = ctypes.c_int64()
        self._chk(lib.qs_query(self.ctx, what, arg, ctypes.byref(v)))
        return v.value

    def close(self):
        if getattr(self, "ctx", None):
            lib.qs_free(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def modes(self):
        kx = np.zeros(self.n_modes)
        ky = np.zeros(self.n_modes)
        self._chk(lib.qs_modes(self.ctx, _dptr(kx), _dptr(ky)))
        return kx, ky

    # -- seeding ----------------------------------------------------------------
    def seed_noise(self, seed: int, amplitude: float):
        self._chk(lib.qs_seed(self.ctx, int(seed) & 0xFFFFFFFFFFFFFFFF, float(amplitude), SEED_NOISE,
                              None, 0, 1))

    def seed_impulse(self, amplitude: float = 1.0):
        self._chk(lib.qs_seed(self.ctx, 0, float(amplitude), SEED_IMPULSE, None, 0, 1))

    def seed_user(self, nb):
        """nb: complex128 [inst][mode][species][xi] concatenated over instances
        (NumPy on the host, or a torch complex128 CUDA tensor)."""
        if isinstance(nb, np.ndarray):
            a = np.ascontiguousarray(nb, np.complex128)
            self._chk(lib.qs_seed(self.ctx, 0, 0.0, SEED_USER, a.ctypes.data_as(ctypes.c_void_p),
                                  a.nbytes, 1))
        else:
            t = nb.contiguous()
            self._chk(lib.qs_seed(self.ctx, 0, 0.0, SEED_USER, ctypes.c_void_p(t.data_ptr()),
                                  t.numel() * t.element_size(), 0))

    def checkpoint(self):
        n = self.query(Q_STATE_BYTES)
        buf = np.empty(n, np.uint8)
        self._chk(lib.qs_diag(self.ctx, DIAG_STATE, buf.ctypes.data_as(ctypes.c_void_p), n, 1))
        return buf

    def restore(self, buf: np.ndarray):
        self._chk(lib.qs_seed(self.ctx, 0, 0.0, SEED_STATE, buf.ctypes.data_as(ctypes.c_void_p),
                              buf.nbytes, 1))

    # -- stepping ---------------------------------------------------------------
    def step(self, n: int = 1):
        self._chk(lib.qs_step(self.ctx, int(n)))

    def step_graph(self, n: int = 1):
        self._chk(lib.qs_step_graph(self.ctx, int(n)))

    def step_green(self, n: int = 1):
        """n steps by the Green's-function path (uniform beams, quiescent front, FP32)."""
        self._chk(lib.qs_step_green(self.ctx, int(n)))

    def sync(self):
        self._chk(lib.qs_sync(self.ctx))

    @property
    def step_count(self):
        return self.query(Q_STEP)

    def launch_count(self):
        return int(lib.qs_launch_count(self.ctx))

    def debug_bounds(self, rows_cut: int):
        self._chk(lib.qs_debug_bounds(self.ctx, int(rows_cut)))

    def debug_waits(self, spin_limit=1 << 24, unsatisfiable=False):
        self._chk(lib.qs_debug_waits(self.ctx, int(spin_limit), 1 if unsatisfiable else 0))

    def set_launch(self, warps_per_cta=2, prefetch=8, persistent=0, ctas_per_sm=8, variant=0, scan_cells=8):
        l = Launch(warps_per_cta, prefetch, persistent, ctas_per_sm, variant, scan_cells)
        self._chk(lib.qs_set_launch(self.ctx, ctypes.byref(l)))

    def get_launch(self):
        l = Launch()
        self._chk(lib.qs_get_launch(self.ctx, ctypes.byref(l)))
        return dict(warps_per_cta=l.warps_per_cta, prefetch=l.prefetch, persistent=l.persistent,
                    ctas_per_sm=l.ctas_per_sm, variant=l.variant, scan_cells=l.scan_cells)

    def tune(self, reps: int = 2, cache_path: str | None = None):
        self._chk(lib.qs_tune(self.ctx, int(reps), cache_path.encode() if cache_path else None))
        return self.get_launch()

    # -- diagnostics --------------------------------------------------------------
    def snapshot_doubles(self, kinds: int) -> int:
        return self.query(Q_SNAPSHOT_BYTES, kinds) // 8

    def record(self, kinds: int, stride: int, n_snap: int):
        """Attach a device record buffer for n_snap snapshots; returns it."""
        torch = self.torch
        if kinds == 0:
            self._chk(lib.qs_record(self.ctx, 0, 1, None, 0))
            self._rec = None
            return None
        buf = torch.empty(n_snap * self.snapshot_doubles(kinds), dtype=torch.float64, device="cuda")
        self._chk(lib.qs_record(self.ctx, kinds, stride, ctypes.c_void_p(buf.data_ptr()),
                                buf.numel() * 8))
        self._rec = (kinds, buf)
        return buf

    def diag(self, kind: int, host: bool = True):
        """One read-only snapshot at the current step (host NumPy or device tensor)."""
        if kind == DIAG_WAKE0:
            n = self.cells * 2
        elif kind == DIAG_XIMAX:
            n = self.cells * 3
        else:
            n = self.snapshot_doubles(kind)
        if host:
            out = np.empty(n, np.float64)
            self._chk(lib.qs_diag(self.ctx, kind, out.ctypes.data_as(ctypes.c_void_p), n * 8, 1))
            return out
        out = self.torch.empty(n, dtype=self.torch.float64, device="cuda")
        self._chk(lib.qs_diag(self.ctx, kind, ctypes.c_void_p(out.data_ptr()), n * 8, 0))
        return out

    # -- layout helpers (host-side reshapes of the library's output layout) ------
    def split_snapshot(self, flat: np.ndarray, kinds: int):
        """Split one snapshot into {'mag': [5][cells][Mp], 'np': complex [cells][Mp],
        'modemax': [3][inst][Mp]}."""
        out, o = {}, 0
        plane = self.cells * self.Mp
        if kinds & REC_MAG:
            out["mag"] = flat[o:o + 5 * plane].reshape(5, self.cells, self.Mp)
            o += 5 * plane
        if kinds & REC_NP:
            out["np"] = flat[o:o + 2 * plane].view(np.complex128).reshape(self.cells, self.Mp)
            o += 2 * plane
        if kinds & REC_MODEMAX:
            out["modemax"] = flat[o:o + 3 * self.n_inst * self.Mp].reshape(3, self.n_inst, self.Mp)
        return out

    def per_instance(self, a: np.ndarray, inst: int, axis: int = -2):
        """Slice instance `inst`'s cells out of a [..., cells, Mp] array and return
        it as [..., mode, xi] (the oracle's order) for the active modes."""
        c0, n = self.cell_off[inst], self.n_xi[inst] if len(self.n_xi) > 1 else self.n_xi[0]
        sl = np.take(a, np.arange(c0, c0 + n), axis=axis)
        sl = np.take(sl, np.arange(self.n_modes), axis=-1)
        return np.swapaxes(sl, -1, -2)

    def state_arrays(self, modes=None):
        """Decode a checkpoint into complex128 n_b and Theta arrays, each
        [inst][mode][species][xi] (the library stores FP32 mantissas m with a
        power-of-two scale W per 32-cell group: value = m * 2**W).
        `modes`: optional index array of active modes to decode (others are
        skipped, which keeps host memory small for large contexts)."""
        raw = self.checkpoint()
        if modes is not None:
            return self._decode_modes(raw, np.asarray(modes))
        hdr = raw[:64].view(np.int64)
        ns, Mp, cells = int(hdr[2]), int(hdr[3]), int(hdr[4])
        body = raw[64:]
        if self.prec == "fp32":
            st = body[:cells * ns * Mp * 16].view(np.float32).reshape(cells, ns, Mp, 4).astype(np.float64)
            ex = body[cells * ns * Mp * 16:].view(np.int32)
            W = (ex >> 8).reshape(-1, Mp).astype(np.int64)
            scale_rows = []
            for i in range(self.n_inst):
                n = self.n_xi[i] if len(self.n_xi) > 1 else self.n_xi[0]
                g0 = sum((self._nxi(k) + 31) // 32 for k in range(i))
                scale_rows.append(W[g0 + np.arange(n) // 32])
            Wc = np.concatenate(scale_rows, axis=0)[:, None, :, None]
            st = np.ldexp(st, Wc)
            nb = st[..., 0] + 1j * st[..., 1]
            th = st[..., 2] + 1j * st[..., 3]
        else:
            half = cells * ns * Mp * 16
            a = body[:half].view(np.float64).reshape(cells, ns, Mp, 2)
            b = body[half:2 * half].view(np.float64).reshape(cells, ns, Mp, 2)
            nb = a[..., 0] + 1j * a[..., 1]
            th = b[..., 0] + 1j * b[..., 1]
        outs = []
        for arr in (nb, th):
            per = []
            for i in range(self.n_inst):
                c0, n = self.cell_off[i], self._nxi(i)
                x = arr[c0:c0 + n, :, :self.n_modes]          # [xi][sp][mode]
                per.append(np.transpose(x, (2, 1, 0)))         # [mode][sp][xi]
            outs.append(per if self.n_inst > 1 else per[0])
        return outs[0], outs[1]

    def _decode_modes(self, raw, sel):
        hdr = raw[:64].view(np.int64)
        ns, Mp, cells = int(hdr[2]), int(hdr[3]), int(hdr[4])
        body = raw[64:]
        if self.prec == "fp32":
            st = body[:cells * ns * Mp * 16].view(np.float32).reshape(cells, ns, Mp, 4)[:, :, sel, :]
            st = st.astype(np.float64)
            W = (body[cells * ns * Mp * 16:].view(np.int32).reshape(-1, Mp)[:, sel] >> 8).astype(np.int64)
            rows = []
            for i in range(self.n_inst):
                g0 = sum((self._nxi(k) + 31) // 32 for k in range(i))
                rows.append(W[g0 + np.arange(self._nxi(i)) // 32])
            st = np.ldexp(st, np.concatenate(rows, axis=0)[:, None, :, None])
            nb, th = st[..., 0] + 1j * st[..., 1], st[..., 2] + 1j * st[..., 3]
        else:
            half = cells * ns * Mp * 16
            a = body[:half].view(np.float64).reshape(cells, ns, Mp, 2)[:, :, sel, :]
            b = body[half:2 * half].view(np.float64).reshape(cells, ns, Mp, 2)[:, :, sel, :]
            nb, th = a[..., 0] + 1j * a[..., 1], b[..., 0] + 1j * b[..., 1]
        outs = []
        for arr in (nb, th):
            per = [np.transpose(arr[self.cell_off[i]:self.cell_off[i] + self._nxi(i)], (2, 1, 0))
                   for i in range(self.n_inst)]
            outs.append(per if self.n_inst > 1 else per[0])
        return outs[0], outs[1]

    def _nxi(self, i):
        return self.n_xi[i] if len(self.n_xi) > 1 else self.n_xi[0]
