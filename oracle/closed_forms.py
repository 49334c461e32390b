"""Closed forms and exact series of the linearised QSA model (test oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).  Each function states
the passage of the paper it restates.  Units are normalised to omega_p, k_p.
"""
from __future__ import annotations

import math
import mpmath as mp
import numpy as np

C_CR = 2.0 / math.sqrt(27.0)   # Appendix B: all saddle roots real iff C < 2/sqrt(27)


def sum_omega2(species, gamma_b: float, shape: float = 1.0) -> float:
    """sum_s omega_bs^2 = sum_s q_s^2 n_bs0 / (m_s gamma_b)   (Sec. II, after Eq. 15)."""
    return sum(q * q * d * shape / (m * gamma_b) for (q, m, d) in species)


def gamma_cfi(sum_w2: float, k2: float) -> float:
    """Temporal CFI rate, Eq. (17): (sum w^2 k^2/(k^2+1))^(1/2)."""
    return math.sqrt(sum_w2 * k2 / (k2 + 1.0))


def gamma_otsi(sum_w2: float, k2: float, gamma_b: float) -> float:
    """Temporal OTSI rate, Eq. (16)."""
    return (math.sqrt(3.0) / 2 ** (4.0 / 3.0)) * sum_w2 ** (1 / 3) * \
        ((k2 + gamma_b ** -2) / (k2 + 1.0)) ** (1 / 3)


def gamma_tsi(sum_w2: float, gamma_b: float) -> float:
    """TSI rate in an unbounded system, Sec. IV.A."""
    return (math.sqrt(3.0) / 2 ** (4.0 / 3.0)) * (sum_w2 / gamma_b ** 2) ** (1 / 3)


def gamma_nbi(sum_w2: float) -> float:
    """Narrow-beam (SMI/HI) rate, Sec. IV.B: Gamma_OTSI(k -> infinity)."""
    return (math.sqrt(3.0) / 2 ** (4.0 / 3.0)) * sum_w2 ** (1 / 3)


def wake_step(xi, rho0: float):
    """Plasma response behind a sharp step of beam charge rho0: Eq. (5) with
    a constant source and a quiescent plasma ahead gives rho0 (1 - cos xi)."""
    return rho0 * (1.0 - np.cos(xi))


def leapfrog_temporal(n, Gamma: float, dt: float):
    """Exact discrete temporal growth of the kick-drift scheme for a
    xi-uniform disturbance (n_p == rho): x_{n+1} - 2x_n + x_{n-1} = (G dt)^2 x_n
    with x_1 = x_0 (1 + (G dt)^2/2) gives x_n = x_0 cosh(n theta),
    cosh(theta) = 1 + (G dt)^2 / 2.  As dt -> 0 the rate theta/dt -> Gamma,
    the temporal CFI rate of Eq. (17)."""
    theta = 2.0 * math.asinh(0.5 * Gamma * dt)
    return np.cosh(np.asarray(n, dtype=np.float64) * theta)


# ---------------------------------------------------------------------------
# Exact impulse response of the per-mode master equation.
# Reduced model, Eq. (18) with a delta(xi)delta(tau) source: its double
# Laplace transform (Eq. 24, written with s = i alpha, p = i beta) is
# 1/(s^2 (p^2+1) - Gamma^2).  Expanding in powers of Gamma^2 and inverting
# term by term (1/s^(2j+2) -> tau^(2j+1)/(2j+1)!;
# (p^2+1)^-(j+1) -> xi^(j+1) j_j(xi) / (2^j j!), j_j the spherical Bessel
# function) gives an everywhere-convergent series.
# Full model (keeps the gamma^-2 d_xi^2 term of Eq. 15 per mode):
# 1/((p^2+1)(s^2+eps) - (Gamma^2+eps)), eps = sum w^2 kappa / gamma^2, so
# 1/s^(2j+2) is replaced by (s^2+eps)^-(j+1) ->
# sqrt(pi)/j! (tau/(2 sqrt eps))^(j+1/2) J_(j+1/2)(sqrt(eps) tau).
# ---------------------------------------------------------------------------
def _xi_factor(j: int, xi):
    # xi^(j+1) j_j(xi) / (2^j j!)
    jj = mp.sqrt(mp.pi / (2 * xi)) * mp.besselj(j + mp.mpf(1) / 2, xi)
    return xi ** (j + 1) * jj / (mp.mpf(2) ** j * mp.factorial(j))


def greens_reduced(tau: float, xi: float, Gamma: float, dps: int = 60, tol=1e-30) -> float:
    """delta n_p(tau, xi) for Eq. (18) with source delta(xi)delta(tau)."""
    if tau <= 0 or xi <= 0:
        return 0.0
    with mp.workdps(dps):
        t, x, G2 = mp.mpf(tau), mp.mpf(xi), mp.mpf(Gamma) ** 2
        total = mp.mpf(0)
        j = 0
        small = 0
        while True:
            term = G2 ** j * t ** (2 * j + 1) / mp.factorial(2 * j + 1) * _xi_factor(j, x)
            total += term
            if abs(term) <= tol * max(abs(total), mp.mpf(1e-300)):
                small += 1
                if small >= 3 and j > x:
                    break
            else:
                small = 0
            j += 1
            if j > 4000:
                raise RuntimeError("series did not converge")
        return float(total)


def greens_full(tau: float, xi: float, Gamma2: float, eps: float, dps: int = 60,
                tol=1e-30) -> float:
    """Impulse response with the gamma^-2 term kept (Eq. 15 per mode):
    (d_xi^2+1) d_tau^2 n + eps d_xi^2 n - Gamma^2 n = delta delta."""
    if tau <= 0 or xi <= 0:
        return 0.0
    with mp.workdps(dps):
        t, x = mp.mpf(tau), mp.mpf(xi)
        G2, e = mp.mpf(Gamma2), mp.mpf(eps)
        a = mp.sqrt(e)
        total = mp.mpf(0)
        j = 0
        small = 0
        while True:
            tj = mp.sqrt(mp.pi) / mp.factorial(j) * (t / (2 * a)) ** (j + mp.mpf(1) / 2) * \
                mp.besselj(j + mp.mpf(1) / 2, a * t)
            term = (G2 + e) ** j * tj * _xi_factor(j, x)
            total += term
            if abs(term) <= tol * max(abs(total), mp.mpf(1e-300)):
                small += 1
                if small >= 3 and j > x:
                    break
            else:
                small = 0
            j += 1
            if j > 4000:
                raise RuntimeError("series did not converge")
        return float(total)


def front_limit_exact(tau, xi, Gamma):
    """Appendix A: exact solution of the front-limit Eq. (19),
    [I0(2 sqrt(G xi tau)) - J0(2 sqrt(G xi tau))] / (2 G)."""
    z = 2.0 * math.sqrt(Gamma * xi * tau)
    return float((mp.besseli(0, z) - mp.besselj(0, z)) / (2 * Gamma))


def front_limit_asym(tau, xi, Gamma):
    """Appendix A, large-argument form: exp(2 sqrt(G xi tau)) /
    (4 sqrt(pi) G (G xi tau)^(1/4))."""
    a = Gamma * xi * tau
    return math.exp(2 * math.sqrt(a)) / (4 * math.sqrt(math.pi) * Gamma * a ** 0.25)


def cfi_st(tau, xi, Gamma):
    """Eq. (28): spatiotemporal CFI near the front (xi << xi_tr)."""
    Gt = Gamma * tau
    return (1 + 3 * xi / (8 * Gt)) * math.exp(2 * math.sqrt(Gt * xi) * (1 - xi / (4 * Gt))) / \
        (4 * math.sqrt(math.pi) * Gamma * (Gt * xi) ** 0.25)


def otsi_st(tau, xi, Gamma):
    """Eq. (29): spatiotemporal OTSI behind the transition (xi >> xi_tr).
    Returns the real value (the bracket plus its complex conjugate)."""
    Gt = Gamma * tau
    pref = (1.0 / (4 * Gamma)) * math.sqrt(2.0 / (3 * math.pi * xi))
    corr = 1 + (1 / 6) * (Gt / xi) ** (2 / 3) * (0.25 + 0.5j * math.sqrt(3))
    ph = 1j * xi + 0.75 * (math.sqrt(3) - 1j) * Gt ** (2 / 3) * xi ** (1 / 3) - 1j * math.pi / 4
    z = corr * np.exp(ph)
    return float(pref * 2 * z.real)


def otsi_st_log_envelope(tau, xi, Gamma):
    """log of the envelope of Eq. (29): leading exponent
    (3 sqrt3 / 4) (G tau)^(2/3) xi^(1/3) = (3/2^(2/3)) G_OTSI tau^(2/3) xi^(1/3)."""
    return 0.75 * math.sqrt(3) * (Gamma * tau) ** (2 / 3) * xi ** (1 / 3)


def cfi_t(tau, Gamma):
    """Eq. (30): observer at xi = xi_tr(tau) = C_cr Gamma tau."""
    Gt = Gamma * tau
    return 3 ** (1 / 6) * math.gamma(1 / 3) / (4 * math.sqrt(2) * math.pi * Gamma * Gt ** (1 / 3)) * \
        math.exp((4 / 3) * math.sqrt(2 / 3) * Gt)


def extended_disturbance_asym(tau, xi, Gamma, S=1.0):
    """Appendix C: tau-asymptotic response to an extended disturbance S,
    S exp(2 sqrt(G xi tau)) / (4 sqrt(pi) (G xi tau)^(1/4))."""
    a = Gamma * xi * tau
    return S * math.exp(2 * math.sqrt(a)) / (4 * math.sqrt(math.pi) * a ** 0.25)


def saddle_roots(C: float):
    """Appendix B, z1..z3: roots of z^3 + z^2 - C^2 = 0 with principal cube
    roots of A.  Reading: the paper prints A = (-2 + 27C^2 + 27C^2 sqrt(C^2 -
    4/27))/2, whose roots do not solve the cubic; Cardano's formula for the
    depressed cubic (z = y - 1/3, y^3 - y/3 + 2/27 - C^2 = 0) gives
    A = (-2 + 27C^2 + 27C sqrt(C^2 - 4/27))/2, used here."""
    C = complex(C)
    A = 0.5 * (-2 + 27 * C ** 2 + 27 * C * np.sqrt(C ** 2 - 4 / 27 + 0j))
    A13 = A ** (1 / 3)
    Am13 = 1 / A13
    s3 = math.sqrt(3)
    z1 = -1 / 3 - (1 - 1j * s3) / 6 * A13 - (1 + 1j * s3) / 6 * Am13
    z2 = -1 / 3 - (1 + 1j * s3) / 6 * A13 - (1 - 1j * s3) / 6 * Am13
    z3 = (1 / 3) * (-1 + A13 + Am13)
    return np.array([z1, z2, z3])
