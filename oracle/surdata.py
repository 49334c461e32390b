"""CPU restatement of the surrogate's training targets (test infrastructure).

From field magnitudes of one mode line at one snapshot (the oracle's
``fields`` output: |dn_b|, |dE|, |dB|, |F_perp|, |E_x| per cell), at cell j:
  y0 = ln(RMS of |dn_b| over the cells within +-1 k_p^-1 of xi_j) - ln A
       (the paper's +-k_p^-1 analysis window, Sec. III.B);
  y1 = 1 (OTSI) if the mode is oscillatory in xi over one plasma wavelength
       around xi_j, else 0 (CFI).  Oscillatory means Re sum conj(Psi) d_xi^2
       Psi < 0: d_xi^2 ~ -1 is the OTSI regime and d_xi^2 >= 0 (growth along
       xi, d_xi^2 << 1 or >> 1) the CFI regimes of Sec. III.A.  With
       d_xi^2 n_p = rho - n_p (Eq. 5), F_perp = i k kappa n_p,
       E_perp = -i k kappa d_xi^2 n_p and B_perp = -i k kappa rho this is
       sum (|F_perp|^2 + |E_perp|^2 - |B_perp|^2) > 0 over the window
       (the magnetic-vs-electric split of the paper's PIC diagnosis).
"""
from __future__ import annotations

import numpy as np


def window(N, dxi, j, half):
    w = max(1, int(round(half / dxi)))
    return max(0, j - w), min(N - 1, j + w)


def targets(mag_line, dxi, j, amplitude):
    """mag_line: [5][N] magnitudes (not logs) of one mode line."""
    nb, E, B, F, Ex = mag_line[0], mag_line[1], mag_line[2], mag_line[3], mag_line[4]
    j0, j1 = window(len(nb), dxi, j, 1.0)
    seg = nb[j0:j1 + 1].astype(np.float64)
    y0 = np.log(np.sqrt(np.mean(seg ** 2))) - np.log(amplitude)
    k0, k1 = window(len(nb), dxi, j, np.pi)
    ep2 = np.maximum(E[k0:k1 + 1] ** 2 - Ex[k0:k1 + 1] ** 2, 0.0)
    s = np.sum(F[k0:k1 + 1] ** 2 + ep2 - B[k0:k1 + 1] ** 2)
    return y0, (1.0 if s > 0 else 0.0)
