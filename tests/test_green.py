"""GPU parity of the Green's-function path (qs_step_green) against the FP64
oracle.  The path is exact for the discrete scheme up to FP32 rounding
(impulse responses from the resident FP32 sweep, convolution in FP32), so it
is held to the FP32 tolerance, against the oracle and against qs_step."""
import numpy as np
import pytest

import oracle
import synth
from test_gpu_parity import FP32_LOG_TOL, GROWTH_CASE, _log_err, _run_oracle, fitted_rates_match

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2607_24234_b300 as m
    return m


def _uniform(n_xi, ks=None, species=None, grid=None, gamma=20.0, dt=1.5, model="full"):
    kw = dict(n_xi=n_xi, dxi=0.05, length=n_xi * 0.05, species=species or [(-1.0, 1.0, 0.05)],
              gamma_b=gamma, dt=dt, model=model, front="quiescent", profile="flattop")
    if grid:
        return synth.scaled(synth.BEAM_3D, nkx=grid, nky=grid, kmax=5.0, **kw)
    return synth.scaled(synth.SLAB_2D, k_list=ks or [0.5, 1.5, 3.0, 6.0], **kw)


@pytest.mark.parametrize("n_xi,grid,species,steps", [
    (150, None, None, 30),
    (700, None, None, 60),                                   # ragged: 88 blocks of 8 cells
    (3000, None, None, 20),                                  # two passes of the CTA over the line
    (200, 16, None, 40),                                     # disc grid: classes of up to 8 modes
    (130, 12, [(-1.0, 1.0, 0.03), (1.0, 1836.0, 0.05)], 25),  # two species
    (256, None, [(-1.0, 1.0, 0.02), (1.0, 1.0, 0.02)], 50),   # pair beam
])
def test_green_noise_seed(qs, n_xi, grid, species, steps):
    p = _uniform(n_xi, species=species, grid=grid)
    s = qs.Solver(p, prec="fp32")
    s.seed_noise(3, 1e-6)
    s.step_green(steps)
    s.sync()
    assert s.step_count == steps
    nb, th = s.state_arrays()
    s.close()
    nb_o, th_o = _run_oracle(p, steps, seed=("noise", 3, 1e-6))
    assert _log_err(nb, nb_o) <= FP32_LOG_TOL and _log_err(th, th_o) <= FP32_LOG_TOL


@pytest.mark.parametrize("species", [None, [(-1.0, 1.0, 0.03), (1.0, 1836.0, 0.05)]])
def test_green_chained_with_theta(qs, species):
    """After ordinary steps Theta is non-zero, so the path also needs the
    responses to Theta impulses; chains of both kinds of calls."""
    p = _uniform(300, species=species, grid=10)
    s = qs.Solver(p, prec="fp32")
    s.seed_noise(4, 1e-6)
    s.step(5)
    s.step_green(17)
    s.step_green(6)
    s.step(4)
    s.sync()
    nb, th = s.state_arrays()
    s.close()
    nb_o, th_o = _run_oracle(p, 32, seed=("noise", 4, 1e-6))
    assert _log_err(nb, nb_o) <= FP32_LOG_TOL and _log_err(th, th_o) <= FP32_LOG_TOL


def test_green_impulse_seed_and_first_step(qs):
    """Impulse seed (Theta only) starting at step 0 (the half kick)."""
    p = _uniform(400, ks=[0.7, 2.0, 4.5])
    s = qs.Solver(p, prec="fp32")
    s.seed_impulse(1.0)
    s.step_green(45)
    s.sync()
    nb, th = s.state_arrays()
    s.close()
    nb_o, th_o = _run_oracle(p, 45, seed=("impulse", 1.0))
    assert _log_err(nb, nb_o) <= FP32_LOG_TOL and _log_err(th, th_o) <= FP32_LOG_TOL


def test_green_matches_step(qs):
    """The same job through qs_step and through qs_step_green."""
    p = _uniform(512, grid=20, gamma=50.0)
    out = []
    for green in (False, True):
        s = qs.Solver(p, prec="fp32")
        s.seed_noise(5, 1e-6)
        (s.step_green if green else s.step)(120)
        s.sync()
        out.append(s.state_arrays())
        s.close()
    assert _log_err(out[1][0], out[0][0]) <= FP32_LOG_TOL and _log_err(out[1][1], out[0][1]) <= FP32_LOG_TOL


def test_green_unsupported(qs):
    base = _uniform(100)
    for p, prec in ((synth.scaled(base, profile="gaussian", sigma_xi=1.0, center_xi=2.5), "fp32"),
                    (synth.scaled(base, front="equilibrium"), "fp32"),
                    (base, "fp64")):
        s = qs.Solver(p, prec=prec)
        s.seed_noise(1, 1e-6)
        with pytest.raises(qs.QSError):
            s.step_green(3)
        s.close()
    s = qs.Solver(base, prec="fp32")
    s.seed_noise(1, 1e-6)
    s.record(qs.REC_MODEMAX, 1, 4)
    with pytest.raises(qs.QSError):
        s.step_green(3)
    s.close()


def test_green_beam3d_full_size_sampled(qs):
    """The benchmark workload at full size (51,468 modes x 2048 cells, 2000
    steps) through the Green's-function path: sampled lines against the
    oracle, every mode through the k/-k pairing of the per-mode maxima."""
    import torch
    p = synth.BEAM_3D
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        s = qs.Solver(p, prec="fp32", stream=st)
        s.seed_noise(0, 1e-6)
        s.step_green(p["n_steps"])
        s.sync()
        mm = s.split_snapshot(s.diag(qs.REC_MODEMAX), qs.REC_MODEMAX)["modemax"][:, 0, :s.n_modes]
        md = oracle.modes(p)
        sel = np.sort(np.random.default_rng(13).choice(s.n_modes, 12, replace=False))
        nb, th = s.state_arrays(modes=sel)
        s.close()
    pos = {int(i): j for j, i in enumerate(md["mode_id"])}
    partner = np.array([pos[int(q)] for q in md["partner_id"]])
    assert np.array_equal(mm, mm[:, partner])
    nb_o, th_o = oracle.seed_noise(p, 0, 1e-6, mode_sel=sel)
    oracle.sweep(p, nb_o, th_o, 0, p["n_steps"], k2=md["k2"][sel])
    assert _log_err(nb, nb_o) <= FP32_LOG_TOL and _log_err(th, th_o) <= FP32_LOG_TOL


def test_fitted_growth_rates_green(qs):
    """Fitted growth rates of the Green's-function path: 40 chained
    qs_step_green calls of 10 steps (after the first, Theta is non-zero, so
    the Theta impulse responses enter too); within 0.5 % of the FP64 oracle."""
    p = synth.scaled(synth.SLAB_2D, **GROWTH_CASE)
    s = qs.Solver(p, prec="fp32")
    s.seed_noise(8, 1e-6)
    fitted_rates_match(lambda k: s.step_green(k), lambda: s.state_arrays()[0])
    s.close()
