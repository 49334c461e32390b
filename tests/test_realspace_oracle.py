"""Pins of the finite-width (real-space) oracle.

- A uniform beam seeded with one transverse Fourier mode cos(k.r) f(xi)
  must evolve exactly as the (pinned) Fourier-mode oracle for |k|: this
  checks the per-point plasma march, the FFT screened-Poisson solve and the
  push together.
- Gaussian beam: the push is a transverse divergence, so the beam charge
  per xi slice is conserved (to spectral accuracy), and a seed symmetric in
  z stays symmetric.
"""
import numpy as np

import oracle
import synth
from oracle import realspace as rs


def _small(**kw):
    p = dict(species=[(-1.0, 1.0, 0.05)], gamma_b=50.0, n_xi=120, dxi=0.05, dt=1.0,
             ny=16, nz=16, Ly=8.0, Lz=8.0, sigma_r=0.8, transverse="gaussian")
    p.update(kw)
    return p


def test_uniform_beam_single_mode_equals_fourier_oracle():
    p = _small(transverse="uniform", ny=16, nz=8, Ly=6.0, Lz=5.0)
    Y, Z = rs.grid(p)
    my, mz = 3, 1
    ky, kz = 2 * np.pi * my / p["Ly"], 2 * np.pi * mz / p["Lz"]
    f = synth.normals(p["n_xi"], 4) * 1e-3
    nb = f[:, None, None] * np.cos(ky * Y + kz * Z)[None]
    G = np.zeros_like(nb)
    steps = 30
    rs.sweep(p, nb, G, 0, steps)
    four = synth.scaled(synth.SLAB_2D, species=p["species"], gamma_b=p["gamma_b"], model="reduced",
                        n_xi=p["n_xi"], dxi=p["dxi"], length=p["n_xi"] * p["dxi"], dt=p["dt"],
                        k_list=[np.hypot(ky, kz)])
    nbf = f.reshape(1, 1, -1).astype(complex)
    thf = np.zeros_like(nbf)
    oracle.sweep(four, nbf, thf, 0, steps)
    expect = nbf[0, 0].real[:, None, None] * np.cos(ky * Y + kz * Z)[None]
    assert np.max(np.abs(nb - expect)) <= 1e-12 * np.max(np.abs(expect))
    # G is n_b0 Theta of the Fourier variables
    expect_g = p["species"][0][2] * thf[0, 0].real[:, None, None] * np.cos(ky * Y + kz * Z)[None]
    assert np.max(np.abs(G - expect_g)) <= 1e-12 * np.max(np.abs(expect_g))


def test_gaussian_beam_conserves_slice_charge_and_symmetry():
    p = _small(ny=32, nz=32)
    noise = synth.normals((p["n_xi"], 32, 32), 7)
    noise = 0.5 * (noise + noise[:, :, ::-1])            # symmetric in z
    nb, G = rs.seed(p, 1e-4, 0.04, noise)
    q0 = nb.sum(axis=(1, 2)).copy()
    rs.sweep(p, nb, G, 0, 25)
    scale = np.max(np.abs(nb.sum(axis=(1, 2))))
    # spectral gradient of Psi against the analytic gradient of n_b0: ~1e-9
    assert np.max(np.abs(nb.sum(axis=(1, 2)) - q0)) <= 1e-7 * max(scale, np.max(np.abs(q0)))
    assert np.max(np.abs(nb - nb[:, :, ::-1])) <= 1e-12 * np.max(np.abs(nb))
    assert np.max(np.abs(G)) > 0
