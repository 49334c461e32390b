"""Replays of the paper's two pair-beam cases with the GPU solver (synthetic
white-noise seeds in place of PIC noise), checked against the paper's
qualitative findings through the CFI/OTSI class rule (pinned separately
against the exact Green's function):

- Sec. III.B (semi-infinite flat top, gamma 2e4, n_b = 0.02 n_p per species,
  k ~ 3, Gamma_CFI tau = 5.63): CFI modulations near the front, oblique OTSI
  modulations further back (the paper: k_p xi <~ 5 and >~ 5; xi_tr = 2.17).
- Sec. III.C (Gaussian, sigma = 3.5 at xi = 15, n_b = 0.03 n_p per species,
  gamma 2000, k ~ 5, front value held, Gamma_CFI tau = 6.43): filaments
  (CFI) ahead of the density peak, longitudinally modulated (OTSI) modes in
  the decreasing ramp, OTSI at k_p xi = 20.
"""
import numpy as np
import pytest

import oracle
import synth
from oracle import closed_forms as cf
from oracle import surdata

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2607_24234_b300 as m
    return m


def _labels(qs, p, steps, seed, xs, held=None, want_mag=False):
    s = qs.Solver(p, prec="fp64", held=held)
    s.seed_noise(seed, 1e-6)
    s.step(steps)
    mag = np.exp(s.per_instance(s.split_snapshot(s.diag(qs.REC_MAG), qs.REC_MAG)["mag"], 0)[:, 0, :])
    s.close()
    lab = np.array([surdata.targets(mag, p["dxi"], int(x / p["dxi"]), 1e-6)[1] for x in xs])
    return (lab, mag) if want_mag else lab


@pytest.mark.parametrize("seed", [0, 1])
def test_semi_infinite_pair_beam(qs, seed):
    sp = [(-1.0, 1.0, 0.02), (1.0, 1.0, 0.02)]
    G = cf.gamma_cfi(cf.sum_omega2(sp, 2e4), 9.0)
    steps = int(round(5.63 / G / 2.0))
    p = synth.scaled(synth.SLAB_2D, species=sp, gamma_b=2e4, n_xi=1000, dxi=0.04, length=40.0, dt=2.0,
                     k_list=[3.0])
    xs = np.arange(0.5, 39.5, 1.0)
    lab = _labels(qs, p, steps, seed, xs)
    assert np.all(lab[xs <= 1.5] == 0)                # CFI ahead of xi_tr = 2.17
    assert np.all(lab[xs >= 5.0] == 1)                # OTSI behind k_p xi ~ 5


@pytest.mark.parametrize("seed", [0, 1])
def test_gaussian_pair_beam_held_front(qs, seed):
    """The front value is held at its initial state (Sec. III.C keeps the
    front value of its window fixed): the plasma at xi = 0 in equilibrium with
    the seeded beam charge of the first cell at tau = 0, P(0) = (rho_0, 0),
    rho_0 = sum_s q_s n_bs(cell 0) of the same Philox noise.  The held value
    enters the solution (the run differs from a zero-held front) and the
    class pattern is the paper's."""
    sp = [(-1.0, 1.0, 0.03), (1.0, 1.0, 0.03)]
    G = cf.gamma_cfi(cf.sum_omega2(sp, 2000.0), 25.0)
    steps = int(round(6.43 / G / 2.0))
    p = synth.scaled(synth.SLAB_2D, species=sp, gamma_b=2000.0, n_xi=1000, dxi=0.03, length=30.0, dt=2.0,
                     k_list=[5.0], profile="gaussian", sigma_xi=3.5, center_xi=15.0, front="held")
    nb0, _ = oracle.seed_noise(p, seed, 1e-6)
    rho0 = sum(q * nb0[0, s, 0] for s, (q, _, _) in enumerate(sp))
    held = np.array([[rho0.real, rho0.imag, 0.0, 0.0]])
    assert np.max(np.abs(held)) > 0.0
    xs = np.arange(0.5, 29.5, 1.0)
    lab, mag = _labels(qs, p, steps, seed, xs, held=held, want_mag=True)
    _, mag0 = _labels(qs, p, steps, seed, xs, held=np.zeros((1, 4)), want_mag=True)
    assert np.max(np.abs(mag - mag0) / np.maximum(mag0, 1e-300)) > 1e-12   # the held value enters
    assert np.all(lab[(xs >= 5.0) & (xs <= 11.0)] == 0)     # filaments ahead of the peak
    assert np.all(lab[xs >= 18.0] == 1)                     # modulated modes in the ramp
    assert lab[np.argmin(np.abs(xs - 20.5))] == 1
