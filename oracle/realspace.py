"""FP64 CPU oracle of the finite-width (transverse real-space) sweep.

TEST INFRASTRUCTURE ONLY.  A beam of finite transverse size n_b0(r_perp)
(Sec. IV.B: narrow beams, self-modulation and hosing) on a periodic
transverse grid; every slow-time step:
  1. plasma response per transverse point: (d_xi^2 + 1) n_p = rho = q n_b
     (Eq. 5, local in r_perp), the exact cell propagator, n_p at cell centres;
  2. per xi slice, the pseudo-potential (grad_perp^2 - 1) Psi = -n_p
     (Eq. 14) by a 2-D FFT: Psi^ = n_p^ / (1 + k^2), and grad_perp Psi by
     spectral derivatives (Nyquist derivative set to zero);
  3. the push of Eqs. (8)-(9) with the transverse divergence kept in
     conservative form and the gamma^-3 term dropped (gamma_b >> 1):
        d_tau G = -(q / (m gamma)) [ n_b0 (Psi - n_p) + grad n_b0 . grad Psi ],
        d_tau n_b = G,
     using grad_perp^2 Psi = Psi - n_p; kick-drift leapfrog, first kick dt/2.
Arrays are [xi][y][z] float64.  numpy.fft serves as the FFT step.
"""
from __future__ import annotations

import numpy as np


def grid(problem):
    ny, nz = int(problem["ny"]), int(problem["nz"])
    Ly, Lz = float(problem["Ly"]), float(problem["Lz"])
    y = (np.arange(ny) + 0.5) * (Ly / ny) - 0.5 * Ly
    z = (np.arange(nz) + 0.5) * (Lz / nz) - 0.5 * Lz
    return np.meshgrid(y, z, indexing="ij")


def profile(problem):
    """n_b0, d_y n_b0, d_z n_b0 on the transverse grid (Gaussian of rms
    sigma_r and peak density_ratio, or uniform)."""
    Y, Z = grid(problem)
    dens = float(problem["species"][0][2])
    if problem.get("transverse", "gaussian") == "uniform":
        nb0 = np.full_like(Y, dens)
        return nb0, np.zeros_like(Y), np.zeros_like(Y)
    s2 = float(problem["sigma_r"]) ** 2
    nb0 = dens * np.exp(-(Y * Y + Z * Z) / (2 * s2))
    return nb0, -(Y / s2) * nb0, -(Z / s2) * nb0


def wavenumbers(n, L):
    """signed spectral indices s = j (j < n/2), j - n (j >= n/2); the
    derivative uses the same with the Nyquist index zeroed."""
    j = np.arange(n)
    s = np.where(j < n // 2, j, j - n).astype(np.float64)
    d = s.copy()
    if n % 2 == 0:
        d[n // 2] = 0.0
    return 2 * np.pi * s / L, 2 * np.pi * d / L


def seed(problem, amplitude, offset, noise=None):
    """n_b = amplitude * (n_b0/peak) * noise + [n_b0(y - offset, z) - n_b0(y, z)]
    on every xi cell (flat-top beam), G = 0.  `noise`: [xi][y][z] standard
    normals (or None for no noise)."""
    N = int(problem["n_xi"])
    nb0, _, _ = profile(problem)
    peak = float(problem["species"][0][2])
    Y, Z = grid(problem)
    shifted = nb0.copy()
    if offset and problem.get("transverse", "gaussian") != "uniform":
        s2 = float(problem["sigma_r"]) ** 2
        shifted = peak * np.exp(-((Y - offset) ** 2 + Z * Z) / (2 * s2))
    base = shifted - nb0
    nb = np.broadcast_to(base, (N,) + base.shape).copy()
    if noise is not None:
        nb += amplitude * (nb0 / peak)[None] * noise
    return nb, np.zeros_like(nb)


def sweep(problem, nb, G, step0, n_steps, record_np=False):
    """Advance (nb, G) in place; returns the last step's n_p and fields
    (Psi, d_y Psi, d_z Psi) at cell centres if record_np."""
    q, m = float(problem["species"][0][0]), float(problem["species"][0][1])
    gam, D, dt = float(problem["gamma_b"]), float(problem["dxi"]), float(problem["dt"])
    N = int(problem["n_xi"])
    c, s, ch, sh = np.cos(D), np.sin(D), np.cos(0.5 * D), np.sin(0.5 * D)
    nb0, gy, gz = profile(problem)
    ky, kyd = wavenumbers(int(problem["ny"]), float(problem["Ly"]))
    kz, kzd = wavenumbers(int(problem["nz"]), float(problem["Lz"]))
    KY, KZ = np.meshgrid(ky, kz, indexing="ij")
    KYd, KZd = np.meshgrid(kyd, kzd, indexing="ij")
    kap = 1.0 / (1.0 + KY * KY + KZ * KZ)
    coef = -q / (m * gam)
    out = None
    for it in range(n_steps):
        h = 0.5 * dt if step0 + it == 0 else dt
        n = np.zeros(nb.shape[1:])
        d = np.zeros_like(n)
        npm = np.empty_like(nb)
        for j in range(N):
            rho = q * nb[j]
            npm[j] = ch * n + sh * d + rho * (1.0 - ch)
            x = c * n + s * d + rho * (1.0 - c)
            d = -s * n + c * d + rho * s
            n = x
        if record_np:
            out = {"np": npm.copy(), "psi": np.empty_like(nb), "dy": np.empty_like(nb), "dz": np.empty_like(nb)}
        for j in range(N):
            F = np.fft.fft2(npm[j])
            P = kap * F
            psi = np.fft.ifft2(P).real
            dpy = np.fft.ifft2(1j * KYd * P).real
            dpz = np.fft.ifft2(1j * KZd * P).real
            S = coef * (nb0 * (psi - npm[j]) + gy * dpy + gz * dpz)
            G[j] += h * S
            nb[j] += dt * G[j]
            if record_np:
                out["psi"][j], out["dy"][j], out["dz"][j] = psi, dpy, dpz
    return out
