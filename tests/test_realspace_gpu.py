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


@pytest.mark.parametrize("n,n_xi,steps", [(64, 80, 20), (256, 24, 6)])
def test_uniform_single_mode(R, n, n_xi, steps):
    """Uniform beam, one transverse Fourier mode: the GPU real-space path
    against the oracle (which equals the pinned Fourier-mode oracle); the
    profile's gradient terms vanish.  N = 64 runs the radix-2 kernels,
    N = 256 the four-step ones."""
    p = _case(n, n_xi, transverse="uniform")
    Y, Z = rs.grid(p)
    mode = np.cos(2 * np.pi * 3 / 8.0 * Y + 2 * np.pi * 2 / 8.0 * Z)
    f = synth.normals(n_xi, 3)
    noise = (f[:, None, None] * mode[None]).astype(np.float32)
    nb_o, G_o = rs.seed(p, 1e-4, 0.0, noise.astype(np.float64))
    rs.sweep(p, nb_o, G_o, 0, steps)
    g = R(p)
    g.seed(amplitude=1e-4, offset=0.0, noise=noise)
    g.step(steps)
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


def test_chunked_launches_at_256(R, monkeypatch):
    """The four-step kernels in chunks of slices (QS_R2_CHUNK = 16: three
    chunks of 16, 16 and 9 slices).  The push kernel stages its half-spectrum
    strips with tensor copies whose row coordinate counts from the chunk's
    first slice.  Chunking changes no arithmetic, so every field equals the
    single-launch run's bit for bit, and both match the oracle."""
    n, n_xi, steps = 256, 41, 2
    p = _case(n, n_xi)
    noise = synth.normals((n_xi, n, n), 11)
    nb_o, G_o = rs.seed(p, 1e-4, 0.04, noise)
    out = rs.sweep(p, nb_o, G_o, 0, steps, record_np=True)
    got = {}
    for chunk in (None, "16"):
        if chunk is None:
            monkeypatch.delenv("QS_R2_CHUNK", raising=False)
        else:
            monkeypatch.setenv("QS_R2_CHUNK", chunk)
        g = R(p)
        g.seed(amplitude=1e-4, offset=0.04, noise=noise.astype(np.float32))
        g.step(steps)
        g.sync()
        got[chunk] = [g.read(w) for w in (0, 1, 2)]
        if chunk is not None:
            assert g.launch_count() == steps * (1 + 3 * 3)   # per step: the march, three chunks of three kernels
        g.close()
    for w, ref in zip((0, 1, 2), (nb_o, G_o, out["np"])):
        assert np.array_equal(got[None][w], got["16"][w]), w
        err = np.max(np.abs(got["16"][w].astype(np.float64) - ref)) / np.max(np.abs(ref))
        assert err <= 1e-3, (w, err)


def test_more_slices_than_one_launch_holds(R):
    """65,600 xi slices, more than the 65,535 a launch's grid holds in y:
    the transform kernels run in two chunks.  Against the oracle after one
    step:
    - n_b matches to 2e-5;
    - G and n_p carry the FP32 march's phase error, which grows linearly
      with the cell count (the rounded cos/sin of dxi turn every cell by the
      same wrong angle): about 3e-4 of the maximum at 65,600 cells, inside
      the FP32 tolerance of 1e-3;
    - the error has no step at the chunk boundary (slice 65,535).
    The radix-2 kernels run here (N = 32); the four-step ones take the same
    chunking."""
    n, n_xi = 32, 65600
    p = _case(n, n_xi)
    noise = synth.normals((n_xi, n, n), 11)
    nb_o, G_o = rs.seed(p, 1e-4, 0.04, noise)
    out = rs.sweep(p, nb_o, G_o, 0, 1, record_np=True)
    g = R(p)
    g.seed(amplitude=1e-4, offset=0.04, noise=noise.astype(np.float32))
    g.step(1)
    g.sync()
    for what, ref, tol in ((0, nb_o, 2e-5), (1, G_o, 1e-3), (2, out["np"], 1e-3)):
        got = g.read(what).astype(np.float64)
        e = np.max(np.abs(got - ref).reshape(n_xi, -1), axis=1) / np.max(np.abs(ref))
        assert e.max() <= tol, (what, e.max())
        before, after = e[65535 - 64:65535].max(), e[65535:65535 + 64].max()
        assert after <= 1.5 * before + 1e-7, (what, before, after)
    assert g.launch_count() == 1 + 2 * 3   # the march, then two chunks of three transform kernels
    g.close()
