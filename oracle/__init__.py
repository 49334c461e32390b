"""FP64 CPU oracle for the linearised quasistatic beam-plasma sweep.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product path
(the CUDA library and its Python binding) never does, and this package never
imports the product.  The C part (``qs_oracle.c``) is a plain sequential loop
over modes, steps and xi cells; ``closed_forms`` holds the paper's analytic
results; ``realspace`` holds the finite-width (transverse grid) oracle.

Every function takes a *problem* dict (see ``synth.workloads``) and NumPy
arrays in the oracle's own layout: ``nb[mode, species, xi]`` and
``th[mode, species, xi]`` complex128.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libqs_oracle.so")
_SRC = os.path.join(_HERE, "qs_oracle.c")

_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP over mode lines)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call([
            "gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
            "-shared", "-fPIC", "-std=c11", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class _Cfg(ctypes.Structure):
    _fields_ = [
        ("n_species", ctypes.c_int),
        ("q", ctypes.c_double * 2), ("m", ctypes.c_double * 2),
        ("dens", ctypes.c_double * 2),
        ("gamma_b", ctypes.c_double),
        ("reduced", ctypes.c_int), ("front", ctypes.c_int),
        ("n_xi", ctypes.c_int), ("dxi", ctypes.c_double), ("dt", ctypes.c_double),
        ("shape", ctypes.POINTER(ctypes.c_double)),
        ("n_modes", ctypes.c_int),
        ("kperp2", ctypes.POINTER(ctypes.c_double)),
        ("held", ctypes.POINTER(ctypes.c_double)),
    ]


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_SO)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int32)
        L.or_profile.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_double, ctypes.c_double, dp]
        L.or_kgrid2.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                ip, dp, dp, dp]
        L.or_philox4x32_10.argtypes = [ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(ctypes.c_uint32),
                                       ctypes.POINTER(ctypes.c_uint32)]
        L.or_seed_noise.argtypes = [ctypes.c_uint64, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                    ctypes.c_int, ctypes.c_int, ip, ip, dp, dp, dp]
        L.or_sweep.argtypes = [ctypes.POINTER(_Cfg), dp, dp, ctypes.c_long, ctypes.c_int,
                               ctypes.c_int, dp, dp]
        L.or_sweep.restype = ctypes.c_int
        L.or_fields.argtypes = [ctypes.POINTER(_Cfg), dp, dp, dp]
        L.or_wake0.argtypes = [ctypes.POINTER(_Cfg), dp, dp]
        L.or_fields_vec.argtypes = [ctypes.POINTER(_Cfg), dp, dp]
        L.or_threads.restype = ctypes.c_int
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def _ip(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)) if a is not None else None


# ---------------------------------------------------------------------------
# Problem geometry (the oracle's own copy of the host-side coefficients)
# ---------------------------------------------------------------------------
PROFILE = {"flattop": 0, "gaussian": 1, "ramp_flattop": 2, "user": 3}


def shape(problem: dict) -> np.ndarray:
    """n_b0(xi_j)/peak at cell centres (flat-top: Sec. II; Gaussian: Sec. III.C)."""
    n = int(problem["n_xi"])
    prof = problem.get("profile", "flattop")
    if prof == "user":
        return np.ascontiguousarray(problem["user_profile"], dtype=np.float64)
    out = np.empty(n, np.float64)
    rc = lib().or_profile(PROFILE[prof], n, float(problem["dxi"]),
                          float(problem.get("length", n * problem["dxi"])),
                          float(problem.get("sigma_xi", 1.0)), float(problem.get("center_xi", 0.0)),
                          float(problem.get("ramp_len", 0.0)), _dp(out))
    if rc != 0:
        raise ValueError(prof)
    return out


def modes(problem: dict):
    """Active transverse modes: dict with k2, kabs, mode_id, partner_id."""
    geom = problem.get("geom", "klist")
    if geom == "klist":
        k = np.asarray(problem["k_list"], np.float64)
        idx = np.arange(len(k), dtype=np.int32)
        return {"k2": k * k, "kabs": np.abs(k), "mode_id": idx, "partner_id": idx.copy(),
                "kx": k.copy(), "ky": np.zeros_like(k)}
    if geom == "kgrid2":
        nkx, nky = int(problem["nkx"]), int(problem["nky"])
        kmax, disc = float(problem["kmax"]), int(problem.get("disc_mask", 1))
        L = lib()
        cnt = L.or_kgrid2(nkx, nky, kmax, disc, None, None, None, None)
        idx = np.empty(cnt, np.int32)
        k2 = np.empty(cnt)
        kx = np.empty(cnt)
        ky = np.empty(cnt)
        L.or_kgrid2(nkx, nky, kmax, disc, _ip(idx), _dp(k2), _dp(kx), _dp(ky))
        ix, iy = idx // nky, idx % nky
        partner = ((nkx - 1 - ix) * nky + (nky - 1 - iy)).astype(np.int32)
        return {"k2": k2, "kabs": np.sqrt(k2), "mode_id": idx, "partner_id": partner,
                "kx": kx, "ky": ky}
    raise ValueError(geom)


def _species(problem):
    sp = problem["species"]
    q = [float(s[0]) for s in sp] + [0.0] * (2 - len(sp))
    m = [float(s[1]) for s in sp] + [1.0] * (2 - len(sp))
    d = [float(s[2]) for s in sp] + [0.0] * (2 - len(sp))
    return len(sp), q, m, d


class _Bound:
    """Keeps the arrays a _Cfg points into alive."""

    def __init__(self, problem, k2=None, held=None):
        self.shape = shape(problem)
        md = modes(problem)
        self.k2 = np.ascontiguousarray(md["k2"] if k2 is None else k2, dtype=np.float64)
        self.held = None if held is None else np.ascontiguousarray(held, dtype=np.float64)
        ns, q, m, d = _species(problem)
        c = _Cfg()
        c.n_species = ns
        c.q[:] = q
        c.m[:] = m
        c.dens[:] = d
        c.gamma_b = float(problem["gamma_b"])
        c.reduced = 1 if problem.get("model", "full") == "reduced" else 0
        c.front = {"quiescent": 0, "equilibrium": 1, "held": 2}[problem.get("front", "quiescent")]
        c.n_xi = int(problem["n_xi"])
        c.dxi = float(problem["dxi"])
        c.dt = float(problem["dt"])
        c.shape = _dp(self.shape)
        c.n_modes = len(self.k2)
        c.kperp2 = _dp(self.k2)
        c.held = _dp(self.held)
        self.cfg = c


def _to_c(a: np.ndarray) -> np.ndarray:
    """complex128 [M,S,N] -> float64 [M,S,N,2] contiguous view/copy."""
    a = np.ascontiguousarray(a, dtype=np.complex128)
    return a.view(np.float64).reshape(a.shape + (2,))


def seed_noise(problem: dict, seed: int, amplitude: float, inst: int = 0, mode_sel=None):
    """White-noise seed (complex Gaussian, Philox4x32-10 counters)."""
    md = modes(problem)
    ids, pids = md["mode_id"], md["partner_id"]
    if mode_sel is not None:
        ids, pids = ids[mode_sel], pids[mode_sel]
    ids = np.ascontiguousarray(ids, np.int32)
    pids = np.ascontiguousarray(pids, np.int32)
    ns = len(problem["species"])
    n = int(problem["n_xi"])
    shp = shape(problem)
    nb = np.zeros((len(ids), ns, n), np.complex128)
    th = np.zeros_like(nb)
    nbv, thv = _to_c(nb), _to_c(th)
    lib().or_seed_noise(int(seed) & 0xFFFFFFFFFFFFFFFF, float(amplitude), int(inst), len(ids), ns, n,
                        _ip(ids), _ip(pids), _dp(shp), _dp(nbv), _dp(thv))
    return nbv.view(np.complex128)[..., 0], thv.view(np.complex128)[..., 0]


def seed_impulse(problem: dict, amplitude: float = 1.0, n_modes=None):
    """Impulse at the front: d_tau rho(tau=0) = amplitude * delta(xi), placed
    in cell 0 of species 0 (the source term of Eq. 23's impulse response)."""
    M = len(modes(problem)["k2"]) if n_modes is None else n_modes
    ns = len(problem["species"])
    n = int(problem["n_xi"])
    q, dens = float(problem["species"][0][0]), float(problem["species"][0][2])
    nb = np.zeros((M, ns, n), np.complex128)
    th = np.zeros_like(nb)
    th[:, 0, 0] = amplitude / (q * dens * shape(problem)[0] * float(problem["dxi"]))
    return nb, th


def sweep(problem: dict, nb: np.ndarray, th: np.ndarray, step0: int, n_steps: int,
          rec_stride: int = 0, record=("mag", "np"), k2=None, held=None):
    """Advance (nb, th) in place by n_steps; optionally record fields.

    Returns dict with 'mag' [snap,5,M,N] (|dn_b|,|dE|,|dB|,|F_perp|,|E_x|) and
    'np' [snap,M,N] complex (n_p at cell centres) when rec_stride > 0.
    """
    b = _Bound(problem, k2=k2, held=held)
    M, N = b.cfg.n_modes, b.cfg.n_xi
    assert nb.shape[0] == M and nb.shape[2] == N
    nbv, thv = _to_c(nb), _to_c(th)
    rec_mag = rec_np = None
    if rec_stride and rec_stride > 0:
        nsnap = (n_steps + rec_stride - 1) // rec_stride
        if "mag" in record:
            rec_mag = np.zeros((nsnap, 5, M, N))
        if "np" in record:
            rec_np = np.zeros((nsnap, M, N, 2))
    rc = lib().or_sweep(ctypes.byref(b.cfg), _dp(nbv), _dp(thv), int(step0), int(n_steps),
                        int(rec_stride or 1), _dp(rec_mag), _dp(rec_np))
    if rc != 0:
        raise ValueError("or_sweep rejected the problem")
    nb[...] = nbv.view(np.complex128)[..., 0]
    th[...] = thv.view(np.complex128)[..., 0]
    out = {}
    if rec_mag is not None:
        out["mag"] = rec_mag
    if rec_np is not None:
        out["np"] = rec_np.view(np.complex128)[..., 0]
    return out


def fields(problem: dict, nb: np.ndarray, k2=None, held=None):
    """Field magnitudes and n_p at the current state (no update)."""
    b = _Bound(problem, k2=k2, held=held)
    M, N = b.cfg.n_modes, b.cfg.n_xi
    nbv = _to_c(nb).copy()
    rec_mag = np.zeros((1, 5, M, N))
    rec_np = np.zeros((1, M, N, 2))
    lib().or_fields(ctypes.byref(b.cfg), _dp(nbv), _dp(rec_mag), _dp(rec_np))
    return {"mag": rec_mag[0], "np": rec_np.view(np.complex128)[0, ..., 0]}


def fields_vec(problem: dict, nb: np.ndarray, k2=None, held=None):
    """Complex field components at the cell centres of the current state:
    dict of [M, N] complex arrays 'ex', 'eperp', 'b', 'fperp' (each the
    coefficient along its transverse unit vector; 2D slab: E_y, B_z, F_y)
    and 'rho' (the beam charge of the cell)."""
    b = _Bound(problem, k2=k2, held=held)
    M, N = b.cfg.n_modes, b.cfg.n_xi
    nbv = _to_c(nb).copy()
    out = np.zeros((M, N, 10))
    lib().or_fields_vec(ctypes.byref(b.cfg), _dp(nbv), _dp(out))
    z = out.view(np.complex128)
    return {"ex": z[..., 0], "eperp": z[..., 1], "b": z[..., 2], "fperp": z[..., 3], "rho": z[..., 4]}


def wake0(problem: dict):
    """Zeroth-order plasma response to the unperturbed beam charge (Eq. 5)."""
    b = _Bound(problem)
    N = b.cfg.n_xi
    edge, mid = np.zeros(N), np.zeros(N)
    lib().or_wake0(ctypes.byref(b.cfg), _dp(edge), _dp(mid))
    return edge, mid


def threads() -> int:
    """OpenMP threads the oracle's parallel loops use."""
    return int(lib().or_threads())


def philox4x32_10(ctr, key):
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (ctypes.c_uint32 * 4)()
    lib().or_philox4x32_10(c, k, o)
    return [int(x) for x in o]
