"""GPU parity: the CUDA sweep (through the C ABI) against the FP64 oracle.

FP64 path: relative error <= 1e-9 per mode line (max-norm and 2-norm).
FP32 + renormalisation path: |ln|x_gpu| - ln|x_ref|| <= 1e-3 on cells with
|x_ref| >= 1e-3 max_xi |x_ref| of their line, fitted growth rates within
0.5%.  Bitwise checks where the arithmetic is identical by construction
(launch shapes, graphs, checkpoints, k/-k pairs).
"""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import closed_forms as cf

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-9
FP32_LOG_TOL = 1e-3


@pytest.fixture(scope="module")
def qs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2607_24234_b300 as m
    return m


def _line_rel(a, b):
    """per mode line: max-norm and 2-norm relative errors over (species, xi)."""
    d = np.abs(a - b).reshape(a.shape[0], -1)
    r = np.abs(b).reshape(b.shape[0], -1)
    mx = np.max(d, axis=1) / np.maximum(np.max(r, axis=1), 1e-300)
    l2 = np.sqrt(np.sum(d * d, axis=1)) / np.maximum(np.sqrt(np.sum(r * r, axis=1)), 1e-300)
    return max(np.max(mx), np.max(l2))


def _log_err(a, b, floor=1e-3):
    """max |ln|a| - ln|b|| over cells with |b| >= floor * line max."""
    A, B = np.abs(a), np.abs(b)
    lm = np.max(B.reshape(B.shape[0], -1), axis=1).reshape((-1,) + (1,) * (B.ndim - 1))
    m = B >= floor * lm
    with np.errstate(divide="ignore"):
        e = np.abs(np.log(A[m]) - np.log(B[m]))
    return float(np.max(e)) if e.size else 0.0


def _run_gpu(qs, problem, prec, steps, seed=("noise", 3, 1e-6), held=None, user=None,
             chunks=None, launch=None):
    s = qs.Solver(problem, prec=prec, held=held)
    if launch:
        s.set_launch(**launch)
    kind = seed[0]
    if kind == "noise":
        s.seed_noise(seed[1], seed[2])
    elif kind == "impulse":
        s.seed_impulse(seed[1])
    else:
        s.seed_user(user)
    for n in (chunks or [steps]):
        s.step(n)
    s.sync()
    nb, th = s.state_arrays()
    return s, nb, th


def _run_oracle(problem, steps, seed=("noise", 3, 1e-6), held=None, user=None, inst=0):
    if seed[0] == "noise":
        nb, th = oracle.seed_noise(problem, seed[1], seed[2], inst=inst)
    elif seed[0] == "impulse":
        nb, th = oracle.seed_impulse(problem, seed[1])
    else:
        nb = np.array(user, dtype=np.complex128)
        th = np.zeros_like(nb)
    oracle.sweep(problem, nb, th, 0, steps, held=held)
    return nb, th


SMALL = [
    # (n_xi, k_list, species, model, front, profile, seed, steps)
    (1, [0.5], [(-1.0, 1.0, 0.05)], "full", "quiescent", "flattop", "noise", 7),
    (2, [1.0, 2.0], [(-1.0, 1.0, 0.05)], "full", "quiescent", "flattop", "noise", 9),
    (31, [0.3, 3.0, 6.0], [(-1.0, 1.0, 0.02)], "reduced", "quiescent", "flattop", "impulse", 40),
    (33, list(np.linspace(0.1, 5, 33)), [(-1.0, 1.0, 0.02)], "full", "equilibrium", "flattop", "noise", 25),
    (65, list(np.linspace(0.2, 4, 70)), [(-1.0, 1.0, 0.03), (1.0, 1.0, 0.03)], "full", "quiescent",
     "gaussian", "noise", 30),
    (100, [0.7, 1.9], [(-1.0, 1.0, 0.03), (1.0, 1836.0, 0.05)], "full", "held", "ramp_flattop", "user", 21),
    (257, list(np.linspace(0.5, 6, 40)), [(-1.0, 1.0, 0.1)], "full", "quiescent", "flattop", "noise", 60),
    # k = 0: the two-stream instability (only the gamma^-3 coupling acts)
    (90, [0.0, 0.0, 1e-3], [(-1.0, 1.0, 0.2)], "full", "quiescent", "flattop", "impulse", 50),
]


def _small_problem(case):
    n_xi, ks, sp, model, front, prof, seed, steps = case
    p = synth.scaled(synth.SLAB_2D, n_xi=n_xi, dxi=0.05, length=n_xi * 0.05 * 0.8, k_list=ks,
                     species=sp, model=model, front=front, profile=prof, gamma_b=20.0, dt=1.5,
                     sigma_xi=0.3 * n_xi * 0.05, center_xi=0.5 * n_xi * 0.05, ramp_len=0.2 * n_xi * 0.05)
    held = None
    if front == "held":
        held = synth.user_seed(len(ks), 1, 2, 11, 1e-4).reshape(len(ks), 2)
        held = np.stack([held.real, held.imag], axis=-1).reshape(len(ks), 4)
    user = None
    if seed == "user":
        user = synth.user_seed(len(ks), len(sp), n_xi, 12, 1e-6)
    sd = {"noise": ("noise", 17, 1e-6), "impulse": ("impulse", 1.0), "user": ("user",)}[seed]
    return p, held, user, sd, steps


@pytest.mark.parametrize("case", SMALL, ids=lambda c: f"nxi{c[0]}-m{len(c[1])}-s{len(c[2])}-{c[3]}-{c[4]}-{c[5]}-{c[6]}")
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_small_cases(qs, case, prec):
    p, held, user, sd, steps = _small_problem(case)
    s, nb, th = _run_gpu(qs, p, prec, steps, seed=sd, held=held, user=user)
    nb_o, th_o = _run_oracle(p, steps, seed=sd, held=held, user=user)
    if prec == "fp64":
        assert _line_rel(nb, nb_o) <= FP64_TOL
        assert _line_rel(th, th_o) <= FP64_TOL
    else:
        assert _log_err(nb, nb_o) <= FP32_LOG_TOL
        assert _log_err(th, th_o) <= FP32_LOG_TOL
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_slab2d_full_size_with_records(qs, prec):
    """The 2D slab workload at full size (64 k x 512 xi x 400 steps), fields
    recorded every 50 steps and once at the end."""
    p = synth.SLAB_2D
    steps, stride = 400, 50
    s = qs.Solver(p, prec=prec)
    s.seed_noise(0, 1e-6)
    kinds = qs.REC_MAG | qs.REC_NP | qs.REC_MODEMAX
    buf = s.record(kinds, stride, steps // stride)
    s.step(steps)
    s.sync()
    fin = s.split_snapshot(s.diag(kinds), kinds)
    rec = buf.cpu().numpy().reshape(steps // stride, -1)
    nb, th = s.state_arrays()
    nb_o, th_o = oracle.seed_noise(p, 0, 1e-6)
    ro = oracle.sweep(p, nb_o, th_o, 0, steps, rec_stride=stride)
    fo = oracle.fields(p, nb_o)
    if prec == "fp64":
        assert _line_rel(nb, nb_o) <= FP64_TOL and _line_rel(th, th_o) <= FP64_TOL
    else:
        assert _log_err(nb, nb_o) <= FP32_LOG_TOL and _log_err(th, th_o) <= FP32_LOG_TOL
    tol = 1e-9 if prec == "fp64" else FP32_LOG_TOL
    for i in range(steps // stride):
        sn = s.split_snapshot(rec[i], kinds)
        mag = s.per_instance(sn["mag"], 0)          # [5][mode][xi] of ln|.|
        npv = s.per_instance(sn["np"], 0)
        for k in range(5):
            ref = ro["mag"][i, k]
            m = ref >= 1e-3 * ref.max(axis=1, keepdims=True)
            assert np.max(np.abs(mag[k][m] - np.log(ref[m]))) <= tol, (i, k)
        if prec == "fp64":
            assert _line_rel(npv, ro["np"][i]) <= FP64_TOL
        else:
            assert _log_err(npv, ro["np"][i]) <= FP32_LOG_TOL
        mm = sn["modemax"][:, 0, :s.n_modes]
        assert np.max(np.abs(mm[0] - np.log(ro["mag"][i, 0].max(axis=1)))) <= tol
    magf = s.per_instance(fin["mag"], 0)
    ref = fo["mag"][0]
    m = ref >= 1e-3 * ref.max(axis=1, keepdims=True)
    assert np.max(np.abs(magf[0][m] - np.log(ref[m]))) <= tol
    s.close()


def test_fp32_renormalisation_survives_extreme_growth(qs):
    """Growth to ~e^150 (past the FP32 range) stays within tolerance thanks
    to the per-(mode, 32-cell) power-of-two exponents."""
    p = synth.scaled(synth.SLAB_2D, n_xi=400, dxi=0.025, length=10.0, species=[(-1.0, 1.0, 0.1)],
                     gamma_b=10.0, k_list=[1.0, 3.0, 6.0, 9.0], dt=2.0)
    steps = 2000
    s, nb, th = _run_gpu(qs, p, "fp32", steps, seed=("noise", 4, 1e-6))
    nb_o, th_o = _run_oracle(p, steps, seed=("noise", 4, 1e-6))
    assert np.max(np.abs(nb_o)) > 1e40      # beyond FP32 range (3.4e38)
    assert _log_err(nb, nb_o) <= FP32_LOG_TOL
    assert _log_err(th, th_o) <= FP32_LOG_TOL
    s.close()


def test_fitted_growth_rates_fp32(qs):
    """Least-squares slope of ln|n_b| vs tau over the last 25% of snapshots at
    fixed (k, xi): FP32 within 0.5% of the FP64 oracle."""
    p = synth.scaled(synth.SLAB_2D, n_xi=256, dxi=0.05, length=12.8, k_list=[1.0, 2.5, 4.0],
                     species=[(-1.0, 1.0, 0.05)], gamma_b=20.0)
    steps, stride = 400, 10
    s = qs.Solver(p, prec="fp32")
    s.seed_noise(8, 1e-6)
    buf = s.record(qs.REC_MAG, stride, steps // stride)
    s.step(steps)
    s.sync()
    rec = buf.cpu().numpy().reshape(steps // stride, -1)
    g = np.stack([s.per_instance(s.split_snapshot(rec[i], qs.REC_MAG)["mag"], 0)[0] for i in
                  range(steps // stride)])                     # [snap][mode][xi] ln|n_b|
    nb_o, th_o = oracle.seed_noise(p, 8, 1e-6)
    ro = oracle.sweep(p, nb_o, th_o, 0, steps, rec_stride=stride)
    o = np.log(ro["mag"][:, 0])
    n = steps // stride
    sel = slice(n - n // 4, n)
    tau = np.arange(n)[sel] * stride * p["dt"]
    for mo in range(3):
        for j in (40, 120, 250):
            rg = np.polyfit(tau, g[sel, mo, j], 1)[0]
            ro_ = np.polyfit(tau, o[sel, mo, j], 1)[0]
            assert abs(rg / ro_ - 1) <= 5e-3, (mo, j, rg, ro_)
    s.close()


GROWTH_CASE = dict(n_xi=256, dxi=0.05, length=12.8, k_list=[1.0, 2.5, 4.0], species=[(-1.0, 1.0, 0.05)],
                   gamma_b=20.0)


def fitted_rates_match(advance, state_nb, steps=400, stride=10, seed=8, tol=5e-3):
    """Fitted growth rates of a GPU path against the FP64 oracle: the path
    advances by `stride` steps per call (advance(stride)) and its state is
    read after every call (state_nb() -> n_b [mode][species][xi]); the oracle
    runs the same chunks.  Least-squares slope of ln|n_b| against tau over the
    last 25 % of the snapshots at fixed (k, xi), relative difference <= tol
    (0.5 %, the FP32 bar)."""
    p = synth.scaled(synth.SLAB_2D, **GROWTH_CASE)
    nb_o, th_o = oracle.seed_noise(p, seed, 1e-6)
    n = steps // stride
    g, o = [], []
    for i in range(n):
        advance(stride)
        oracle.sweep(p, nb_o, th_o, i * stride, stride)
        g.append(np.log(np.abs(state_nb()[:, 0, :])))
        o.append(np.log(np.abs(nb_o[:, 0, :])))
    g, o = np.array(g), np.array(o)
    sel = slice(n - n // 4, n)
    tau = (np.arange(n)[sel] + 1) * stride * p["dt"]
    worst = 0.0
    for mo in range(3):
        for j in (40, 120, 250):
            rg = np.polyfit(tau, g[sel, mo, j], 1)[0]
            ro_ = np.polyfit(tau, o[sel, mo, j], 1)[0]
            worst = max(worst, abs(rg / ro_ - 1))
    assert worst <= tol, worst
    return worst


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_kgrid_pairs_conjugate_bitwise(qs, prec):
    p = synth.scaled(synth.BEAM_3D, nkx=16, nky=16, kmax=4.0, n_xi=96, dxi=0.05, length=4.8)
    s, nb, th = _run_gpu(qs, p, prec, 30, seed=("noise", 21, 1e-6))
    md = oracle.modes(p)
    kx, ky = s.modes()
    assert np.array_equal(kx, md["kx"]) and np.array_equal(ky, md["ky"])
    pos = {int(i): j for j, i in enumerate(md["mode_id"])}
    for j, pi in enumerate(md["partner_id"]):
        jj = pos[int(pi)]
        assert np.array_equal(nb[j], np.conj(nb[jj])) and np.array_equal(th[j], np.conj(th[jj]))
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_launch_shapes_and_graph_bitwise(qs, prec):
    """Every launch shape and the CUDA-graph path run the same per-line
    arithmetic, so they agree bit for bit; so does a checkpoint resume."""
    import torch
    p = synth.scaled(synth.BEAM_3D, nkx=24, nky=24, kmax=5.0, n_xi=150, dxi=0.04, length=6.0)
    ref = None
    U = (4, 8) if prec == "fp32" else (2, 4)
    shapes = [dict(warps_per_cta=w, prefetch=u, persistent=pers, ctas_per_sm=4, variant=0)
              for w in (1, 2, 4, 8) for u in U for pers in (0, 1)]
    C = (8, 16) if prec == "fp32" else (4, 8)
    shapes += [dict(warps_per_cta=1, prefetch=cc, persistent=pers, ctas_per_sm=cps, variant=1)
               for cc in C for pers, cps in ((0, 8), (1, 8), (1, 32))]
    for sh in shapes:
        s_, nb, th = _run_gpu(qs, p, prec, 13, seed=("noise", 2, 1e-6), launch=sh)
        s_.close()
        if ref is None:
            ref = (nb, th)
        assert np.array_equal(nb, ref[0]) and np.array_equal(th, ref[1]), sh
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        s = qs.Solver(p, prec=prec, stream=st)
        s.seed_noise(2, 1e-6)
        s.step_graph(5)
        s.step_graph(4)
        s.step_graph(4)
        s.sync()
        nb, th = s.state_arrays()
        assert np.array_equal(nb, ref[0]) and np.array_equal(th, ref[1])
        s.close()
    # checkpoint after 6 steps, resume for 7 more
    s = qs.Solver(p, prec=prec)
    s.seed_noise(2, 1e-6)
    s.step(6)
    ck = s.checkpoint()
    s.step(3)
    s.restore(ck)
    assert s.step_count == 6
    s.step(7)
    s.sync()
    nb, th = s.state_arrays()
    assert np.array_equal(nb, ref[0]) and np.array_equal(th, ref[1])
    s.close()


def test_batched_uneven_instances_fp64(qs):
    """Several instances with different densities, gamma, lengths and n_xi
    in one persistent launch; each instance against its own oracle run."""
    insts = synth.batch_instances(6, param_seed=3, base=synth.scaled(synth.BATCH_BASE, nkx=8, nky=8),
                                  dxi=0.5)
    s = qs.Solver(insts, prec="fp64")
    s.set_launch(warps_per_cta=1, prefetch=4, persistent=1, ctas_per_sm=2)
    s.seed_noise(0, 1e-6)
    s.step(25)
    s.sync()
    nb, th = s.state_arrays()
    for i, p in enumerate(insts):
        nb_o, th_o = oracle.seed_noise(p, 0, 1e-6, inst=i)
        oracle.sweep(p, nb_o, th_o, 0, 25)
        assert _line_rel(nb[i], nb_o) <= FP64_TOL, i
        assert _line_rel(th[i], th_o) <= FP64_TOL, i
    s.close()


def test_greens_function_on_gpu(qs):
    """Impulse response on the GPU (FP64) against the exact series of the
    paper's Green's function (same discretisation error as the oracle)."""
    n0, gam, k, D = 0.08, 2.0, 1000.0, 0.05
    G = math.sqrt(n0 / gam * k * k / (1 + k * k))
    p = synth.scaled(synth.SLAB_2D, species=[(-1.0, 1.0, n0)], gamma_b=gam, model="reduced",
                     n_xi=100, dxi=D, length=5.0, dt=D, k_list=[k])
    s = qs.Solver(p, prec="fp64")
    s.seed_impulse(1.0)
    s.step(500)
    npv = s.per_instance(s.split_snapshot(s.diag(qs.REC_NP), qs.REC_NP)["np"], 0)[0]
    xs = [1.0, 2.0, 3.0, 4.0]
    ex = np.array([cf.greens_reduced(25.0, x, G) for x in xs])
    got = npv[[int(round(x / D)) for x in xs]].real
    assert np.max(np.abs(got / ex - 1)) < 6e-4
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_temporal_cfi_cosh_law(qs, prec):
    ks = [0.5, 2.0, 5.0]
    p = synth.scaled(synth.SLAB_2D, front="equilibrium", n_xi=64, dxi=0.05, length=3.2, k_list=ks,
                     gamma_b=50.0)
    user = np.ones((3, 1, 64), complex) * (0.3 + 0.4j) * 1e-6
    s, nb, th = _run_gpu(qs, p, prec, 300, seed=("user",), user=user)
    w2 = cf.sum_omega2(p["species"], p["gamma_b"])
    tol = 1e-11 if prec == "fp64" else 1e-4
    for i, k in enumerate(ks):
        ex = user[i, 0] * cf.leapfrog_temporal(300, cf.gamma_cfi(w2, k * k), p["dt"])
        assert np.max(np.abs(nb[i, 0] / ex - 1)) < tol
    s.close()


def test_wake0_matches_closed_form(qs):
    p = synth.scaled(synth.SLAB_2D, n_xi=800, dxi=0.05, length=40.0)
    s = qs.Solver(p, prec="fp64")
    w = s.diag(qs.DIAG_WAKE0).reshape(-1, 2)
    xe = (np.arange(800) + 1) * 0.05
    xm = (np.arange(800) + 0.5) * 0.05
    assert np.max(np.abs(w[:, 0] - cf.wake_step(xe, -0.01))) < 1e-14
    assert np.max(np.abs(w[:, 1] - cf.wake_step(xm, -0.01))) < 1e-14
    s.close()


def test_nonfinite_detected_and_cleared(qs):
    p = synth.scaled(synth.SLAB_2D, n_xi=64, k_list=[1.0, 2.0])
    s = qs.Solver(p, prec="fp32")
    bad = synth.user_seed(2, 1, 64, 1, 1e-6)
    bad[1, 0, 40] = np.nan
    s.seed_user(bad)
    s.step(2)
    with pytest.raises(qs.QSError) as e:
        s.sync()
    assert e.value.status == qs.QS_ERR_NONFINITE
    with pytest.raises(qs.QSError) as e:
        s.step(1)
    assert e.value.status == qs.QS_ERR_STATE
    s.seed_noise(1, 1e-6)
    s.step(2)
    s.sync()
    s.close()


def test_record_overflow_rejected(qs):
    p = synth.scaled(synth.SLAB_2D, n_xi=64, k_list=[1.0, 2.0])
    s = qs.Solver(p, prec="fp32")
    s.seed_noise(1, 1e-6)
    s.record(qs.REC_MAG, 2, 3)          # room for steps 0, 2, 4
    s.step(5)
    with pytest.raises(qs.QSError) as e:
        s.step(2)                       # would write snapshot 3
    assert e.value.status == qs.QS_ERR_ARG
    s.record(0, 1, 0)
    s.step(2)
    s.sync()
    s.close()


def test_autotuner_cache_roundtrip(qs, tmp_path):
    p = synth.scaled(synth.BEAM_3D, nkx=32, nky=32, kmax=6.0, n_xi=256, dxi=0.05, length=12.8)
    s = qs.Solver(p, prec="fp32")
    s.seed_noise(3, 1e-6)
    before = s.state_arrays()
    cache = str(tmp_path / "tune.json")
    best = s.tune(reps=2, cache_path=cache)
    after = s.state_arrays()
    assert np.array_equal(before[0], after[0]) and np.array_equal(before[1], after[1])
    assert s.step_count == 0
    txt = open(cache).read()
    assert "fp32-ns1" in txt
    s2 = qs.Solver(p, prec="fp32")
    s2.seed_noise(3, 1e-6)
    assert s2.tune(reps=2, cache_path=cache) == best
    s.close()
    s2.close()


@pytest.mark.slow
def test_batched_512_instances_full_size_sampled(qs):
    """The batched workload at full size: 512 instances (n_b/n_p, gamma, L
    drawn with seed 0; 200..8000 cells at dxi = 0.025), the 64 x 64 disc grid
    (3,228 modes), 1000 steps, FP32, one persistent LPT launch.  Checked on
    sampled (instance, mode) lines against the oracle through the per-mode
    maxima over xi of ln|n_b|, ln|dE|, ln|dB|, and on every mode through the
    k/-k pairing (bitwise equal maxima)."""
    insts = synth.batch_instances(512, param_seed=0)
    steps = 1000
    s = qs.Solver(insts, prec="fp32")
    assert s.n_modes == 3228
    s.seed_noise(0, 1e-6)
    s.step(steps)
    s.sync()
    mm = s.split_snapshot(s.diag(qs.REC_MODEMAX), qs.REC_MODEMAX)["modemax"][:, :, :s.n_modes]
    assert np.all(np.isfinite(mm))
    md = oracle.modes(insts[0])
    pos = {int(i): j for j, i in enumerate(md["mode_id"])}
    partner = np.array([pos[int(p)] for p in md["partner_id"]])
    assert np.array_equal(mm, mm[:, :, partner])
    rng = np.random.default_rng(5)
    lens = np.array([p["n_xi"] for p in insts])
    picks = [int(np.argmax(lens)), int(np.argmin(lens))] + list(rng.choice(512, 10, replace=False))
    worst = 0.0
    for i in picks:
        p = insts[i]
        sel = rng.choice(s.n_modes, 2, replace=False)
        nb, th = oracle.seed_noise(p, 0, 1e-6, inst=i, mode_sel=sel)
        oracle.sweep(p, nb, th, 0, steps, k2=md["k2"][sel])
        f = oracle.fields(p, nb, k2=md["k2"][sel])
        ref = np.log(np.max(f["mag"][[0, 1, 2]], axis=2))      # [3][2 modes]
        got = mm[:, i, sel]
        worst = max(worst, float(np.max(np.abs(got - ref))))
    assert worst <= 1e-3, worst
    s.close()


@pytest.mark.parametrize("S,V", [(2, 1), (4, 5), (8, 16), (32, 3)])
@pytest.mark.parametrize("case", [SMALL[0], SMALL[2], SMALL[3], SMALL[5], SMALL[6]],
                         ids=lambda c: f"nxi{c[0]}-m{len(c[1])}-s{len(c[2])}-{c[4]}")
def test_scan_variant_fp64(qs, case, S, V):
    """FP64 chunked-scan variant (lanes split xi, shuffle scan of the cell
    propagators) against the oracle at 1e-9."""
    p, held, user, sd, steps = _small_problem(case)
    s, nb, th = _run_gpu(qs, p, "fp64", steps, seed=sd, held=held, user=user,
                         launch=dict(warps_per_cta=2, prefetch=S, persistent=0, ctas_per_sm=8, variant=2,
                                     scan_cells=V))
    nb_o, th_o = _run_oracle(p, steps, seed=sd, held=held, user=user)
    assert _line_rel(nb, nb_o) <= FP64_TOL
    assert _line_rel(th, th_o) <= FP64_TOL
    s.close()


def test_scan_variant_slab2d_full_size(qs):
    """The 2D slab workload (64 modes x 512 cells x 400 steps, FP64): the
    scan variant against the oracle, and its time against thread-per-line."""
    import torch
    p = synth.SLAB_2D
    nb_o, th_o = oracle.seed_noise(p, 0, 1e-6)
    oracle.sweep(p, nb_o, th_o, 0, 400)
    times = {}
    for name, launch in (("line", dict(warps_per_cta=1, prefetch=4, persistent=0, ctas_per_sm=8, variant=1)),
                         ("scan", dict(warps_per_cta=1, prefetch=32, persistent=0, ctas_per_sm=8, variant=2,
                                       scan_cells=4))):
        s = qs.Solver(p, prec="fp64")
        s.set_launch(**launch)
        s.seed_noise(0, 1e-6)
        s.step(2)
        s.seed_noise(0, 1e-6)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        s.step(400)
        e1.record()
        s.sync()
        times[name] = e0.elapsed_time(e1)
        nb, th = s.state_arrays()
        assert _line_rel(nb, nb_o) <= FP64_TOL and _line_rel(th, th_o) <= FP64_TOL
        s.close()
    print({"slab2d_fp64_ms": times})
    assert times["scan"] < times["line"]


def test_bounded_wait_timeout_reported_and_recovered(qs):
    """Failure detection without a fault: the TMA kernel's tile barriers are
    made to expect more bytes than their copies deliver; every wait runs out
    after a short bound, the kernel reports QS_ERR_TIMEOUT and returns, and
    the context works again after the hook is cleared and the state reseeded."""
    p = synth.scaled(synth.SLAB_2D, n_xi=64, k_list=[0.5, 1.5, 3.0])
    s = qs.Solver(p, prec="fp32")
    s.set_launch(warps_per_cta=1, prefetch=8, persistent=0, ctas_per_sm=8, variant=1)
    s.seed_noise(3, 1e-6)
    s.debug_waits(spin_limit=2000, unsatisfiable=True)
    s.step(1)
    with pytest.raises(qs.QSError) as e:
        s.sync()
    assert e.value.status == qs.QS_ERR_TIMEOUT
    s.debug_waits()
    s.seed_noise(3, 1e-6)
    s.step(10)
    s.sync()
    nb, th = s.state_arrays()
    nb_o, th_o = _run_oracle(p, 10, seed=("noise", 3, 1e-6))
    assert _log_err(nb, nb_o) <= FP32_LOG_TOL
    s.close()


def test_per_xi_maxima_and_persistent_graph(qs):
    """Per-xi maxima over modes against the oracle's fields, and CUDA-graph
    stepping of a batched persistent launch against plain stepping."""
    import torch
    p = synth.scaled(synth.BEAM_3D, nkx=20, nky=20, kmax=5.0, n_xi=100, dxi=0.05, length=5.0)
    s = qs.Solver(p, prec="fp64")
    s.seed_noise(6, 1e-6)
    s.step(30)
    xm = s.diag(qs.DIAG_XIMAX).reshape(3, -1)
    nb_o, th_o = oracle.seed_noise(p, 6, 1e-6)
    oracle.sweep(p, nb_o, th_o, 0, 30)
    f = oracle.fields(p, nb_o)["mag"]
    ref = np.log(np.max(f[[0, 1, 2]], axis=1))          # [3][xi]
    assert np.max(np.abs(xm - ref)) <= 1e-9
    s.close()
    insts = synth.batch_instances(5, param_seed=4, base=synth.scaled(synth.BATCH_BASE, nkx=8, nky=8), dxi=0.5)
    st = torch.cuda.Stream()
    outs = []
    for graph in (False, True):
        with torch.cuda.stream(st):
            s = qs.Solver(insts, prec="fp32", stream=st)
            s.set_launch(warps_per_cta=1, prefetch=8, persistent=1, ctas_per_sm=2, variant=1)
            s.seed_noise(2, 1e-6)
            for _ in range(3):
                (s.step_graph if graph else s.step)(4)
            s.sync()
            outs.append(s.state_arrays())
            s.close()
    for i in range(5):
        assert np.array_equal(outs[0][0][i], outs[1][0][i]) and np.array_equal(outs[0][1][i], outs[1][1][i])


@pytest.mark.slow
@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_beam3d_full_size_sampled(qs, prec):
    """The benchmark workload at full size in the launch shape bench.py uses
    (tuned): 51,468 modes x 2048 cells x 2000 steps.  Sampled mode lines
    against the oracle; every mode through the k/-k pairing of the per-mode
    maxima (bitwise equal)."""
    import torch
    p = synth.BEAM_3D
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        s = qs.Solver(p, prec=prec, stream=st)
        s.seed_noise(0, 1e-6)
        s.tune(reps=64)          # the trial length bench.py tunes with
        s.step(p["n_steps"])
        s.sync()
        mm = s.split_snapshot(s.diag(qs.REC_MODEMAX), qs.REC_MODEMAX)["modemax"][:, 0, :s.n_modes]
        md = oracle.modes(p)
        sel = np.sort(np.random.default_rng(11).choice(s.n_modes, 12, replace=False))
        nb, th = s.state_arrays(modes=sel)
        s.close()
    pos = {int(i): j for j, i in enumerate(md["mode_id"])}
    partner = np.array([pos[int(q)] for q in md["partner_id"]])
    assert np.array_equal(mm, mm[:, partner])
    nb_o, th_o = oracle.seed_noise(p, 0, 1e-6, mode_sel=sel)
    oracle.sweep(p, nb_o, th_o, 0, p["n_steps"], k2=md["k2"][sel])
    if prec == "fp64":
        assert _line_rel(nb, nb_o) <= FP64_TOL and _line_rel(th, th_o) <= FP64_TOL
    else:
        assert _log_err(nb, nb_o) <= FP32_LOG_TOL and _log_err(th, th_o) <= FP32_LOG_TOL


def test_host_diag_staging_reuse(qs):
    """Host-form snapshots share one staging buffer per context, grown when a
    larger kind is asked for: small, large, small again, each equal to the
    device-form snapshot of the same step (the entries of real modes; the
    padding modes' entries are not written)."""
    p, held, user, sd, steps = _small_problem(max(SMALL, key=lambda c: c[0] * len(c[1])))
    s, _, _ = _run_gpu(qs, p, "fp32", 3, seed=sd, held=held, user=user)
    M = len(p["k_list"])
    for kind in (qs.REC_MODEMAX, qs.REC_MAG | qs.REC_NP, qs.REC_MODEMAX, qs.REC_MAG):
        h = s.split_snapshot(s.diag(kind, host=True), kind)
        d = s.split_snapshot(s.diag(kind, host=False).cpu().numpy(), kind)
        assert h.keys() == d.keys()
        for key in h:
            assert np.array_equal(h[key][..., :M], d[key][..., :M]), (kind, key)
    s.close()
