"""GPU parity of the finite-width real-space sweep against its FP64 oracle
(reduced sizes, every FFT size), and invariants at full size."""
import numpy as np
import pytest

import synth
from oracle import realspace as rs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2607_24234_b300.realspace import RealSpace
    return RealSpace


def _case(n, n_xi, **kw):
    p = dict(species=[(-1.0, 1.0, 0.05)], gamma_b=50.0, n_xi=n_xi, dxi=0.05, dt=1.0, ny=n, nz=n,
             Ly=8.0, Lz=8.0, sigma_r=0.8, transverse="gaussian")
    p.update(kw)
    return p


@pytest.mark.parametrize("n,n_xi,steps", [(32, 120, 25), (64, 37, 9), (128, 9, 4), (256, 5, 3), (256, 41, 2)])
def test_matches_oracle(R, n, n_xi, steps):
    p = _case(n, n_xi)
    noise = synth.normals((n_xi, n, n), 11)
    nb_o, G_o = rs.seed(p, 1e-4, 0.04, noise)
    out = rs.sweep(p, nb_o, G_o, 0, steps, record_np=True)
    g = R(p)
    g.seed(amplitude=1e-4, offset=0.04, noise=noise.astype(np.float32))
    g.step(steps)
    g.sync()
    for what, ref in ((0, nb_o), (1, G_o), (2, out["np"])):
        got = g.read(what).astype(np.float64)
        err = np.max(np.abs(got - ref)) / np.max(np.abs(ref))
        assert err <= 2e-5, (what, err)
    g.close()


def test_uniform_single_mode(R):
    """Uniform beam, one transverse Fourier mode: the GPU real-space path
    against the oracle (which equals the pinned Fourier-mode oracle)."""
    p = _case(64, 80, transverse="uniform")
    Y, Z = rs.grid(p)
    mode = np.cos(2 * np.pi * 3 / 8.0 * Y + 2 * np.pi * 2 / 8.0 * Z)
    f = synth.normals(80, 3)
    noise = (f[:, None, None] * mode[None]).astype(np.float32)
    nb_o, G_o = rs.seed(p, 1e-4, 0.0, noise.astype(np.float64))
    rs.sweep(p, nb_o, G_o, 0, 20)
    g = R(p)
    g.seed(amplitude=1e-4, offset=0.0, noise=noise)
    g.step(20)
    got = g.read(0).astype(np.float64)
    assert np.max(np.abs(got - nb_o)) / np.max(np.abs(nb_o)) <= 2e-5
    g.close()


@pytest.mark.slow
def test_narrow_beam_full_size_invariants(R):
    """The narrow-beam workload at full transverse and xi size for a few
    steps: finite, and the beam charge of every slice is conserved by the
    divergence-form push (relative to the seed's slice charge scale)."""
    p = synth.NARROW_BEAM
    g = R(p)
    g.seed(seed=0, amplitude=p["amplitude"], offset=p["offset"])
    q0 = g.read(0).astype(np.float64).sum(axis=(1, 2))
    g.step(20)
    g.sync()
    nb = g.read(0).astype(np.float64)
    assert np.all(np.isfinite(nb))
    drift = np.max(np.abs(nb.sum(axis=(1, 2)) - q0))
    scale = np.max(np.abs(nb).sum(axis=(1, 2)))
    assert drift <= 1e-4 * scale
    assert g.launch_count() == 80
    g.close()


@pytest.mark.parametrize("n,n_xi", [(32, 20), (256, 5)])
def test_nonfinite_state_reported(R, n, n_xi):
    """A NaN in one seeded cell reaches the fields through the transverse
    solve and the push writes non-finite values; the push's check reports
    it at the next sync (QS_ERR_NONFINITE), and a clean reseed clears it.
    Covers the radix-2 kernels (N = 32) and the four-step ones (N = 256)."""
    from paper_2607_24234_b300 import QSError
    p = _case(n, n_xi)
    noise = synth.normals((n_xi, n, n), 5).astype(np.float32)
    g = R(p)
    g.seed(amplitude=1e-4, offset=0.04, noise=noise)
    g.step(2)
    g.sync()                      # finite: no error
    bad = noise.copy()
    bad[n_xi // 2, n // 3, n // 5] = np.nan
    g.seed(amplitude=1e-4, offset=0.04, noise=bad)
    g.step(2)
    with pytest.raises(QSError) as ei:
        g.sync()
    assert ei.value.status == 5
    g.seed(amplitude=1e-4, offset=0.04, noise=noise)
    g.step(2)
    g.sync()
    g.close()
