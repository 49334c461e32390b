"""Seeded synthetic workloads shared by the tests, the benchmark and the oracle.

This module holds problem *descriptions* and seeded random inputs only; it
contains none of the model's arithmetic (no coefficients, no k-grid
construction, no profiles, no propagators).  Both the CUDA path and the CPU
oracle derive everything else from these plain dicts on their own.

Problem dict keys
-----------------
species      list of (q, m, density_ratio) per beam species (1 or 2)
gamma_b      beam Lorentz factor
model        "full" | "reduced"   (keep / drop the gamma^-3 term)
front        "quiescent" | "equilibrium" | "held"
profile      "flattop" | "gaussian" | "ramp_flattop" | "user"
length, sigma_xi, center_xi, ramp_len, user_profile
n_xi, dxi, dt
geom         "klist" (k_list) | "kgrid2" (nkx, nky, kmax, disc_mask)
"""
from __future__ import annotations

import copy
import numpy as np

# --- the paper's cases as synthetic workloads --------------------------------
# 2D slab: one electron-like species (q=-1, m=1), n_b/n_p = 0.01, gamma = 1000,
# sharp front, flat top of length 20; 64 transverse k in (0, 4]; 512 xi cells;
# 400 steps of dt = 2; white noise 1e-6 (seed 0).
SLAB_2D = dict(
    name="slab2d_64k_512xi_400steps",
    species=[(-1.0, 1.0, 0.01)], gamma_b=1000.0, model="full", front="quiescent",
    profile="flattop", length=20.0, n_xi=512, dxi=20.0 / 512, dt=2.0,
    geom="klist", k_list=[4.0 * (i + 1) / 64 for i in range(64)],
    n_steps=400, seed=0, amplitude=1e-6,
)

# 3D uniform beam: 256 x 256 (kx, ky) grid over |k| <= 6 (disc), 2048 cells
# over a length of 100, 2000 steps of dt = 2.
BEAM_3D = dict(
    name="beam3d_256sq_disc_2048xi_2000steps",
    species=[(-1.0, 1.0, 0.01)], gamma_b=1000.0, model="full", front="quiescent",
    profile="flattop", length=100.0, n_xi=2048, dxi=100.0 / 2048, dt=2.0,
    geom="kgrid2", nkx=256, nky=256, kmax=6.0, disc_mask=1,
    n_steps=2000, seed=0, amplitude=1e-6,
)

# Batched sweep: instances share a 64 x 64 disc grid (|k| <= 6), dxi = 0.025,
# 1000 steps; per-instance n_b/n_p ~ 10^U(-3,-1), gamma ~ 10^U(1,4),
# length ~ U(5, 200) (so 200..8000 cells).
BATCH_BASE = dict(
    name="batch_64sq_disc",
    species=[(-1.0, 1.0, 0.01)], gamma_b=1000.0, model="full", front="quiescent",
    profile="flattop", length=100.0, n_xi=4000, dxi=0.025, dt=2.0,
    geom="kgrid2", nkx=64, nky=64, kmax=6.0, disc_mask=1,
    n_steps=1000, seed=0, amplitude=1e-6,
)


# Finite-width narrow beam (self-modulation / hosing): one electron species,
# Gaussian transverse profile of rms 0.5 and peak n_b/n_p = 0.05, gamma =
# 2e4, flat top of length 400 (16,000 cells), periodic 256 x 256 transverse
# grid over +-8 sigma_r, 500 steps; seeded by a 0.01 sigma_r centroid offset
# plus white noise 1e-6 (relative to the local density).
NARROW_BEAM = dict(
    name="narrow_beam_256sq_16000xi_500steps",
    species=[(-1.0, 1.0, 0.05)], gamma_b=2.0e4, n_xi=16000, dxi=0.025, dt=2.0,
    ny=256, nz=256, Ly=8.0, Lz=8.0, sigma_r=0.5, transverse="gaussian",
    n_steps=500, seed=0, amplitude=1e-6, offset=0.005,
)


def batch_instances(n_inst: int = 512, param_seed: int = 0, base: dict | None = None,
                    dxi: float = 0.025):
    """Seeded parameter draw for the batched sweep (reading: NumPy PCG64 with
    `param_seed`; noise seed of instance i is i)."""
    base = copy.deepcopy(BATCH_BASE if base is None else base)
    rng = np.random.Generator(np.random.PCG64(param_seed))
    lnb = rng.uniform(-3.0, -1.0, n_inst)
    lg = rng.uniform(1.0, 4.0, n_inst)
    L = rng.uniform(5.0, 200.0, n_inst)
    out = []
    for i in range(n_inst):
        p = copy.deepcopy(base)
        p["species"] = [(-1.0, 1.0, float(10.0 ** lnb[i]))]
        p["gamma_b"] = float(10.0 ** lg[i])
        n_xi = int(round(L[i] / dxi))
        p["n_xi"] = n_xi
        p["dxi"] = dxi
        p["length"] = n_xi * dxi
        p["inst_seed"] = i
        out.append(p)
    return out


def scaled(problem: dict, **kw) -> dict:
    """Copy of a problem with some keys replaced (smaller parity cases)."""
    p = copy.deepcopy(problem)
    p.update(kw)
    return p


def normals(shape, seed: int):
    """Standard normals (NumPy PCG64) for seeds passed in as data."""
    return np.random.Generator(np.random.PCG64(seed)).standard_normal(shape)


def user_seed(n_modes: int, n_species: int, n_xi: int, seed: int, amplitude: float):
    """Complex Gaussian array [mode, species, xi] (NumPy PCG64), for seeds
    passed in as data (USER seeds) rather than drawn by either side."""
    rng = np.random.Generator(np.random.PCG64(seed))
    a = rng.standard_normal((n_modes, n_species, n_xi, 2))
    return (amplitude / np.sqrt(2.0)) * (a[..., 0] + 1j * a[..., 1])
