"""GPU parity of the resident (on-chip) FP32 sweep against the FP64 oracle.

The resident variant keeps every line in registers for all steps of a call
and joins xi with a block scan of the cell propagators, so its rounding
differs from the streaming kernels: it is held to the FP32 tolerance against
the oracle, and bit for bit only where the arithmetic is the same by
construction (graph replay, chunked calls, k/-k pairs).
"""
import numpy as np
import pytest

import oracle
import synth
from test_gpu_parity import (FP32_LOG_TOL, GROWTH_CASE, SMALL, _log_err, _run_gpu, _run_oracle, _small_problem,
                             fitted_rates_match)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2607_24234_b300 as m
    return m


def _res(V=8, w=4, pers=0, cps=2, regs=False):
    return dict(warps_per_cta=w, prefetch=V, persistent=pers, ctas_per_sm=cps, variant=3, scan_cells=1 if regs else 8)


def _fits(n_xi, V, w):
    return ((-(-n_xi // V) + 31) // 32) * 32 <= 32 * w


@pytest.mark.parametrize("case", SMALL, ids=lambda c: f"nxi{c[0]}-m{len(c[1])}-s{len(c[2])}-{c[3]}-{c[4]}-{c[5]}-{c[6]}")
@pytest.mark.parametrize("V", [8, 16, 32])
def test_small_cases_resident(qs, case, V):
    p, held, user, sd, steps = _small_problem(case)
    ns = len(p["species"])
    if V == 32 and ns == 2:
        pytest.skip("32 cells per thread is for one species")
    ok = (lambda w: w in (2, 4, 8)) if V == 32 else (lambda w: w in (4, 8, 16)) if (V == 16 and ns == 2) else (lambda w: True)
    w = next(w for w in (1, 2, 4, 8, 16) if _fits(p["n_xi"], V, w) and ok(w) and w >= 2)
    s, nb, th = _run_gpu(qs, p, "fp32", steps, seed=sd, held=held, user=user, launch=_res(V, w))
    nb_o, th_o = _run_oracle(p, steps, seed=sd, held=held, user=user)
    assert _log_err(nb, nb_o) <= FP32_LOG_TOL
    assert _log_err(th, th_o) <= FP32_LOG_TOL
    s.close()


@pytest.mark.parametrize("n_xi,V,w,pers", [
    (700, 8, 8, 0),      # 88 -> 96 threads per line: 2 lines per 256-thread CTA, 64 idle threads
    (700, 8, 8, 1),
    (1000, 16, 2, 1),    # 63 -> 64 threads, one line per CTA
    (33, 16, 4, 0),      # 3 -> 32 threads: 4 lines per CTA, most threads without cells
    (2048, 16, 4, 1),    # the benchmark's line length
    (2048, 32, 4, 1),    # Theta in shared memory, 2 lines per CTA
    (1000, 32, 8, 0),    # 32 -> 32 threads: 4 lines per CTA
])
def test_ragged_packing(qs, n_xi, V, w, pers):
    """Lines per CTA, idle threads and a mode count that is not a multiple
    of the lines per CTA."""
    p = synth.scaled(synth.SLAB_2D, n_xi=n_xi, dxi=0.05, length=n_xi * 0.05, k_list=list(np.linspace(0.3, 5.0, 37)),
                     species=[(-1.0, 1.0, 0.05)], gamma_b=20.0, dt=1.5)
    steps = 40
    s, nb, th = _run_gpu(qs, p, "fp32", steps, seed=("noise", 5, 1e-6), launch=_res(V, w, pers))
    nb_o, th_o = _run_oracle(p, steps, seed=("noise", 5, 1e-6))
    assert _log_err(nb, nb_o) <= FP32_LOG_TOL and _log_err(th, th_o) <= FP32_LOG_TOL
    s.close()


def test_batched_instances_resident(qs):
    """Instances of different length, density and gamma in one persistent
    launch (LPT order); each against its own oracle run."""
    insts = synth.batch_instances(6, param_seed=4, base=synth.scaled(synth.BATCH_BASE, nkx=8, nky=8), dxi=0.25)
    s = qs.Solver(insts, prec="fp32")
    mx = max(p["n_xi"] for p in insts)
    w = next(w for w in (1, 2, 4, 8, 16) if _fits(mx, 8, w))
    s.set_launch(**_res(16, max(w, 4), 1, 2))
    s.seed_noise(0, 1e-6)
    s.step(30)
    s.sync()
    nb, th = s.state_arrays()
    for i, p in enumerate(insts):
        nb_o, th_o = oracle.seed_noise(p, 0, 1e-6, inst=i)
        oracle.sweep(p, nb_o, th_o, 0, 30)
        assert _log_err(nb[i], nb_o) <= FP32_LOG_TOL, i
        assert _log_err(th[i], th_o) <= FP32_LOG_TOL, i
    s.close()


def test_records_split_the_call(qs):
    """A call that records every 7 steps: the recording steps run the
    register kernel, the others stay on chip; snapshots and final state
    against the oracle."""
    p = synth.scaled(synth.SLAB_2D, n_xi=300, dxi=0.05, length=15.0, k_list=[0.5, 1.5, 3.0, 6.0],
                     species=[(-1.0, 1.0, 0.05)], gamma_b=20.0)
    steps, stride = 50, 7
    s = qs.Solver(p, prec="fp32")
    s.set_launch(**_res(32, 2))
    s.seed_noise(6, 1e-6)
    n_snap = (steps - 1) // stride + 1
    buf = s.record(qs.REC_MAG | qs.REC_NP, stride, n_snap)
    s.step(steps)
    s.sync()
    rec = buf.cpu().numpy().reshape(n_snap, -1)
    nb, th = s.state_arrays()
    nb_o, th_o = oracle.seed_noise(p, 6, 1e-6)
    ro = oracle.sweep(p, nb_o, th_o, 0, steps, rec_stride=stride)
    assert _log_err(nb, nb_o) <= FP32_LOG_TOL and _log_err(th, th_o) <= FP32_LOG_TOL
    for i in range(n_snap):
        sn = s.split_snapshot(rec[i], qs.REC_MAG | qs.REC_NP)
        mag = s.per_instance(sn["mag"], 0)
        for k in range(5):
            ref = ro["mag"][i, k]
            m = ref >= 1e-3 * ref.max(axis=1, keepdims=True)
            assert np.max(np.abs(mag[k][m] - np.log(ref[m]))) <= FP32_LOG_TOL, (i, k)
        assert _log_err(s.per_instance(sn["np"], 0), ro["np"][i]) <= FP32_LOG_TOL
    s.close()


def test_extreme_growth_resident(qs):
    """Growth to ~e^150, past the FP32 range: per-thread exponents."""
    p = synth.scaled(synth.SLAB_2D, n_xi=400, dxi=0.025, length=10.0, species=[(-1.0, 1.0, 0.1)],
                     gamma_b=10.0, k_list=[1.0, 3.0, 6.0, 9.0], dt=2.0)
    steps = 2000
    s, nb, th = _run_gpu(qs, p, "fp32", steps, seed=("noise", 4, 1e-6), launch=_res(32, 2))
    nb_o, th_o = _run_oracle(p, steps, seed=("noise", 4, 1e-6))
    assert np.max(np.abs(nb_o)) > 1e40
    assert _log_err(nb, nb_o) <= FP32_LOG_TOL and _log_err(th, th_o) <= FP32_LOG_TOL
    s.close()


def test_resident_bitwise_properties(qs):
    """Chunked calls (exponents are powers of two, so re-entering a line at
    another scale changes no bits), graph replay, and k/-k conjugate pairs."""
    import torch
    p = synth.scaled(synth.BEAM_3D, nkx=24, nky=24, kmax=5.0, n_xi=150, dxi=0.04, length=6.0)
    L = _res(32, 4)
    _, nb, th = _run_gpu(qs, p, "fp32", 13, seed=("noise", 2, 1e-6), launch=L)
    _, nb2, th2 = _run_gpu(qs, p, "fp32", 13, seed=("noise", 2, 1e-6), launch=L, chunks=[6, 1, 6])
    assert np.array_equal(nb, nb2) and np.array_equal(th, th2)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        s = qs.Solver(p, prec="fp32", stream=st)
        s.set_launch(**L)
        s.seed_noise(2, 1e-6)
        for n in (5, 4, 4):
            s.step_graph(n)
        s.sync()
        nb3, th3 = s.state_arrays()
        s.close()
    assert np.array_equal(nb, nb3) and np.array_equal(th, th3)
    md = oracle.modes(p)
    pos = {int(i): j for j, i in enumerate(md["mode_id"])}
    for j, pi in enumerate(md["partner_id"]):
        jj = pos[int(pi)]
        assert np.array_equal(nb[j], np.conj(nb[jj])) and np.array_equal(th[j], np.conj(th[jj]))
    nb_o, th_o = _run_oracle(p, 13, seed=("noise", 2, 1e-6))
    assert _log_err(nb, nb_o) <= FP32_LOG_TOL and _log_err(th, th_o) <= FP32_LOG_TOL


def test_launch_validation(qs):
    p = synth.scaled(synth.SLAB_2D, n_xi=2048, dxi=0.05, length=102.4, k_list=[1.0, 2.0])
    s = qs.Solver(p, prec="fp32")
    with pytest.raises(qs.QSError):
        s.set_launch(**_res(8, 4))      # 256 threads per line, CTA of 128
    s.set_launch(**_res(16, 4))
    s.close()
    s = qs.Solver(p, prec="fp64")
    with pytest.raises(qs.QSError):
        s.set_launch(**_res(16, 4))     # FP32 only
    s.close()


def test_beam3d_full_size_sampled_resident(qs):
    """The benchmark workload at full size (51,468 modes x 2048 cells x 2000
    steps in one call) in the benchmark's tuned shape (32 cells per thread,
    64-thread CTAs): sampled mode lines against the oracle, and every mode
    through the k/-k pairing of the per-mode maxima (bitwise)."""
    import torch
    p = synth.BEAM_3D
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        s = qs.Solver(p, prec="fp32", stream=st)
        s.set_launch(**_res(32, 2))
        s.seed_noise(0, 1e-6)
        s.step(p["n_steps"])
        s.sync()
        mm = s.split_snapshot(s.diag(qs.REC_MODEMAX), qs.REC_MODEMAX)["modemax"][:, 0, :s.n_modes]
        md = oracle.modes(p)
        sel = np.sort(np.random.default_rng(12).choice(s.n_modes, 12, replace=False))
        nb, th = s.state_arrays(modes=sel)
        s.close()
    pos = {int(i): j for j, i in enumerate(md["mode_id"])}
    partner = np.array([pos[int(q)] for q in md["partner_id"]])
    assert np.array_equal(mm, mm[:, partner])
    nb_o, th_o = oracle.seed_noise(p, 0, 1e-6, mode_sel=sel)
    oracle.sweep(p, nb_o, th_o, 0, p["n_steps"], k2=md["k2"][sel])
    assert _log_err(nb, nb_o) <= FP32_LOG_TOL and _log_err(th, th_o) <= FP32_LOG_TOL


@pytest.mark.parametrize("n_xi,V,w,species", [
    (700, 32, 2, [(-1.0, 1.0, 0.05)]),                      # one warp per line, ragged tail
    (2100, 32, 4, [(-1.0, 1.0, 0.05)]),                     # three warps per line (cross-warp maximum)
    (300, 16, 4, [(-1.0, 1.0, 0.03), (1.0, 1836.0, 0.05)]),  # two species, Theta in shared memory
])
def test_modemax_on_chip(qs, n_xi, V, w, species):
    """Per-mode maxima of |dn_b|, |dE|, |dB| recorded every 7 steps inside
    the resident kernel, and a read-only maxima pass at the end, against the
    oracle's fields (maxima over the real cells only)."""
    p = synth.scaled(synth.SLAB_2D, n_xi=n_xi, dxi=0.05, length=n_xi * 0.05, k_list=[0.5, 1.5, 3.0, 6.0],
                     species=species, gamma_b=20.0, dt=1.5)
    steps, stride = 40, 7
    n_snap = (steps - 1) // stride + 1
    s = qs.Solver(p, prec="fp32")
    s.set_launch(**_res(V, w))
    s.seed_noise(9, 1e-6)
    buf = s.record(qs.REC_MODEMAX, stride, n_snap)
    n0 = s.launch_count()
    s.step(steps)
    s.sync()
    assert s.launch_count() - n0 == 1          # no split: the maxima are taken on chip
    rec = buf.cpu().numpy().reshape(n_snap, -1)
    s.record(0, 1, 0)
    fin = s.split_snapshot(s.diag(qs.REC_MODEMAX), qs.REC_MODEMAX)["modemax"][:, 0, :s.n_modes]
    mms = [s.split_snapshot(rec[i], qs.REC_MODEMAX)["modemax"][:, 0, :s.n_modes] for i in range(n_snap)]
    s.close()
    nb_o, th_o = oracle.seed_noise(p, 9, 1e-6)
    ro = oracle.sweep(p, nb_o, th_o, 0, steps, rec_stride=stride)
    fo = oracle.fields(p, nb_o)
    for i, mm in enumerate(mms):
        for k in range(3):
            assert np.max(np.abs(mm[k] - np.log(ro["mag"][i, k].max(axis=1)))) <= FP32_LOG_TOL, (i, k)
    for k in range(3):
        assert np.max(np.abs(fin[k] - np.log(fo["mag"][k].max(axis=1)))) <= FP32_LOG_TOL, k


@pytest.mark.parametrize("pers", [0, 1])
def test_batched_exact_cta_sizes(qs, pers):
    """Instances whose lines need 1 .. 8 warps at 32 cells per thread: one
    launch per CTA size (256: 8, 4 or 1 lines; 192: 2 or 1; 160; 224), each
    CTA a whole number of lines; every instance against its own oracle run."""
    lengths = [1000, 2000, 3000, 5000, 6000, 7000, 8000]
    base = synth.scaled(synth.BATCH_BASE, nkx=8, nky=8, dxi=0.025)
    insts = []
    for i, n in enumerate(lengths):
        insts.append(synth.scaled(base, n_xi=n, length=n * 0.025, inst_seed=i,
                                  species=[(-1.0, 1.0, 0.02 + 0.01 * i)], gamma_b=30.0 + 10 * i))
    s = qs.Solver(insts, prec="fp32")
    s.set_launch(**_res(32, 8, pers, 2))
    s.seed_noise(0, 1e-6)
    n0 = s.launch_count()
    s.step(8)
    s.sync()
    assert s.launch_count() - n0 == 4        # CTA sizes 160, 192, 224, 256
    nb, th = s.state_arrays()
    s.close()
    for i, p in enumerate(insts):
        nb_o, th_o = oracle.seed_noise(p, 0, 1e-6, inst=i)
        oracle.sweep(p, nb_o, th_o, 0, 8)
        assert _log_err(nb[i], nb_o) <= FP32_LOG_TOL, i
        assert _log_err(th[i], th_o) <= FP32_LOG_TOL, i


@pytest.mark.parametrize("n_xi,V,ks", [
    (1, 8, [1.3]),            # one cell, one mode: thread 0 alone, 31 idle lanes
    (256, 8, [0.4, 2.2]),     # exactly one warp of 8-cell chunks
    (257, 8, [0.4, 2.2]),     # one cell into a second warp
    (1024, 32, [5.0]),        # one warp of 32-cell chunks, shared-memory Theta
    (1025, 32, [5.0]),
])
def test_resident_edges(qs, n_xi, V, ks):
    p = synth.scaled(synth.SLAB_2D, n_xi=n_xi, dxi=0.05, length=n_xi * 0.05, k_list=ks,
                     species=[(-1.0, 1.0, 0.05)], gamma_b=20.0, dt=1.5)
    w = next(w for w in (2, 4, 8) if _fits(n_xi, V, w))
    s, nb, th = _run_gpu(qs, p, "fp32", 25, seed=("noise", 7, 1e-6), launch=_res(V, w))
    nb_o, th_o = _run_oracle(p, 25, seed=("noise", 7, 1e-6))
    assert _log_err(nb, nb_o) <= FP32_LOG_TOL and _log_err(th, th_o) <= FP32_LOG_TOL
    s.close()


def test_resident_held_front_on_zero_state(qs):
    """A held front driving an all-zero state: the line starts without any
    exponent except the front's (thread 0), the others take theirs from the
    line maximum."""
    ks = [0.6, 1.7, 3.1]
    p = synth.scaled(synth.SLAB_2D, n_xi=600, dxi=0.05, length=30.0, k_list=ks, front="held",
                     species=[(-1.0, 1.0, 0.05)], gamma_b=20.0, dt=1.5)
    held = synth.user_seed(len(ks), 1, 2, 21, 1e-3).reshape(len(ks), 2)
    held = np.stack([held.real, held.imag], axis=-1).reshape(len(ks), 4)
    zero = np.zeros((len(ks), 1, 600), complex)
    s, nb, th = _run_gpu(qs, p, "fp32", 30, seed=("user",), held=held, user=zero, launch=_res(32, 2))
    nb_o, th_o = _run_oracle(p, 30, seed=("user",), held=held, user=zero)
    assert np.max(np.abs(nb_o)) > 0
    assert _log_err(nb, nb_o) <= FP32_LOG_TOL and _log_err(th, th_o) <= FP32_LOG_TOL
    s.close()


def test_resident_nonfinite_detected(qs):
    p = synth.scaled(synth.SLAB_2D, n_xi=64, k_list=[1.0, 2.0])
    s = qs.Solver(p, prec="fp32")
    s.set_launch(**_res(16, 2))
    bad = synth.user_seed(2, 1, 64, 1, 1e-6)
    bad[1, 0, 40] = np.nan
    s.seed_user(bad)
    s.step(3)
    with pytest.raises(qs.QSError) as e:
        s.sync()
    assert e.value.status == qs.QS_ERR_NONFINITE
    s.seed_noise(1, 1e-6)
    s.step(2)
    s.sync()
    s.close()


@pytest.mark.parametrize("V,w", [(32, 2), (8, 1)])
def test_fitted_growth_rates_resident(qs, V, w):
    """Fitted growth rates (last 25 % of 40 snapshots over 400 steps) of the
    resident kernel itself: every 10-step call is one on-chip launch, the
    state is read back between calls; within 0.5 % of the FP64 oracle."""
    p = synth.scaled(synth.SLAB_2D, **GROWTH_CASE)
    s = qs.Solver(p, prec="fp32")
    s.set_launch(**_res(V, w))
    s.seed_noise(8, 1e-6)
    n0 = s.launch_count()
    fitted_rates_match(lambda k: s.step(k), lambda: s.state_arrays()[0])
    assert s.launch_count() - n0 == 40          # one resident launch per call, nothing else
    s.close()


# Theta in registers at the largest cells per thread (32 of one species, 16 of
# two): the same arithmetic as the shared-memory form, in another storage
@pytest.mark.parametrize("case", SMALL, ids=lambda c: f"nxi{c[0]}-m{len(c[1])}-s{len(c[2])}-{c[3]}-{c[4]}-{c[5]}-{c[6]}")
def test_small_cases_resident_theta_registers(qs, case):
    p, held, user, sd, steps = _small_problem(case)
    V = 32 if len(p["species"]) == 1 else 16
    w = next(w for w in (1, 2, 4, 8) if _fits(p["n_xi"], V, w))
    s, nb, th = _run_gpu(qs, p, "fp32", steps, seed=sd, held=held, user=user, launch=_res(V, w, regs=True))
    nb_o, th_o = _run_oracle(p, steps, seed=sd, held=held, user=user)
    assert _log_err(nb, nb_o) <= FP32_LOG_TOL
    assert _log_err(th, th_o) <= FP32_LOG_TOL
    s.close()


@pytest.mark.parametrize("n_xi,V,w,pers,species", [
    (700, 32, 8, 0, None),      # 22 -> 32 threads per line: 8 lines per 256-thread CTA
    (2048, 32, 2, 1, None),     # the benchmark's line length, one line per CTA
    (2100, 32, 4, 0, None),     # 66 -> 96 threads: 3 warps, cross-warp prefix
    (1000, 16, 4, 1, [(-1.0, 1.0, 0.03), (1.0, 1836.0, 0.05)]),
])
def test_theta_registers_packing_and_bitwise(qs, n_xi, V, w, pers, species):
    """Ragged packing, and bit-identity with the shared-memory form (same
    operations in the same order) and across chunked calls."""
    sp = species or [(-1.0, 1.0, 0.05)]
    p = synth.scaled(synth.SLAB_2D, n_xi=n_xi, dxi=0.05, length=n_xi * 0.05, k_list=list(np.linspace(0.3, 5.0, 37)),
                     species=sp, gamma_b=20.0, dt=1.5)
    steps = 40
    s, nb, th = _run_gpu(qs, p, "fp32", steps, seed=("noise", 5, 1e-6), launch=_res(V, w, pers, regs=True))
    s.close()
    nb_o, th_o = _run_oracle(p, steps, seed=("noise", 5, 1e-6))
    assert _log_err(nb, nb_o) <= FP32_LOG_TOL and _log_err(th, th_o) <= FP32_LOG_TOL
    ws = next(x for x in (2, 4, 8, 16) if _fits(n_xi, V, x) and (x >= 4 or len(sp) == 1))
    s2, nb2, th2 = _run_gpu(qs, p, "fp32", steps, seed=("noise", 5, 1e-6), launch=_res(V, ws, pers))
    s2.close()
    assert np.array_equal(nb, nb2) and np.array_equal(th, th2)
    s3, nb3, th3 = _run_gpu(qs, p, "fp32", steps, seed=("noise", 5, 1e-6), launch=_res(V, w, pers, regs=True),
                            chunks=[17, 1, 22])
    s3.close()
    assert np.array_equal(nb, nb3) and np.array_equal(th, th3)


def test_renormalisation_interval_from_growth_bound(qs):
    """The context takes the resident sweep's renormalisation interval from
    qs_growth_bound: a dense, slow beam checks every 8 steps (and still
    matches the oracle over a fast-growing run); a problem whose bound leaves
    no interval refuses the resident variant and the Green's-function path."""
    p = synth.scaled(synth.SLAB_2D, species=[(-1.0, 1.0, 0.1)], gamma_b=10.0, dt=2.0, n_xi=4000, dxi=0.05,
                     length=200.0, k_list=[0.5, 2.0, 6.0])
    g, ev = qs.growth_bound(p)
    assert ev == 8
    steps = 120
    s, nb, th = _run_gpu(qs, p, "fp32", steps, seed=("noise", 6, 1e-6), launch=_res(32, 4))
    assert s.query(qs.Q_RES_EVERY) == 8
    s.close()
    nb_o, th_o = _run_oracle(p, steps, seed=("noise", 6, 1e-6))
    assert np.max(np.abs(nb_o)) > 1e6 * 1e-6            # the run grows
    assert _log_err(nb, nb_o) <= FP32_LOG_TOL and _log_err(th, th_o) <= FP32_LOG_TOL
    bad = synth.scaled(synth.SLAB_2D, species=[(-1.0, 1.0, 100.0)], gamma_b=1.1, dt=1000.0, n_xi=4000, dxi=0.25,
                       length=1000.0, k_list=[1.0])
    assert qs.growth_bound(bad)[1] == 0
    s = qs.Solver(bad, prec="fp32")
    assert s.query(qs.Q_RES_EVERY) == 0
    with pytest.raises(qs.QSError) as e:
        s.set_launch(**_res(32, 8))
    assert e.value.status == qs.QS_ERR_UNSUPPORTED
    s.seed_noise(1, 1e-6)
    with pytest.raises(qs.QSError) as e:
        s.step_green(1)
    assert e.value.status == qs.QS_ERR_UNSUPPORTED
    s.close()


def test_uniform_weight_kernel(qs, monkeypatch):
    """Uniform profile whose lines fill whole warps (1024 cells, 32 per
    thread): the resident kernel that holds the cell weight in a register
    against the one that reads per-cell weights, bit for bit, and against the
    FP64 oracle; 40 steps include renormalisation checks."""
    p = synth.scaled(synth.SLAB_2D, n_xi=1024, dxi=0.05, length=1024 * 0.05, k_list=[0.3, 0.9, 1.7, 2.6],
                     profile="flattop", gamma_b=20.0, dt=1.5)
    out = {}
    for env in ("0", "1"):
        monkeypatch.setenv("QS_RES_NO_UNIFORM", env)
        s, nb, th = _run_gpu(qs, p, "fp32", 40, seed=("noise", 5, 1e-6), launch=_res(32, 2))
        out[env] = (nb, th)
        s.close()
    assert np.array_equal(out["0"][0], out["1"][0]) and np.array_equal(out["0"][1], out["1"][1])
    nb_o, th_o = _run_oracle(p, 40, seed=("noise", 5, 1e-6))
    assert _log_err(out["0"][0], nb_o) <= FP32_LOG_TOL
    assert _log_err(out["0"][1], th_o) <= FP32_LOG_TOL


@pytest.mark.parametrize("n_xi,w", [(1000, 2), (1100, 2), (257, 2), (33, 2)])
def test_uniform_weight_ragged_lines(qs, monkeypatch, n_xi, w):
    """Uniform profile whose lines end inside a thread's chunk: the
    register-weight kernel lets the cells past the end evolve (they feed only
    later padding cells and are never written), the per-cell-weight kernel
    keeps them at zero.  Both against the FP64 oracle, and against each other
    at rounding level (only the end thread's renormalisation sees the
    padding); 60 steps include renormalisation checks and a growth of about
    e^6."""
    p = synth.scaled(synth.SLAB_2D, n_xi=n_xi, dxi=0.05, length=n_xi * 0.05, k_list=[0.3, 0.9, 1.7, 2.6],
                     profile="flattop", gamma_b=20.0, dt=1.5)
    out = {}
    for env in ("0", "1"):
        monkeypatch.setenv("QS_RES_NO_UNIFORM", env)
        s, nb, th = _run_gpu(qs, p, "fp32", 60, seed=("noise", 7, 1e-6), launch=_res(32, w))
        out[env] = (nb, th)
        s.close()
    nb_o, th_o = _run_oracle(p, 60, seed=("noise", 7, 1e-6))
    for env in ("0", "1"):
        assert _log_err(out[env][0], nb_o) <= FP32_LOG_TOL, env
        assert _log_err(out[env][1], th_o) <= FP32_LOG_TOL, env
    assert _log_err(out["0"][0], out["1"][0]) <= 1e-5
    assert _log_err(out["0"][1], out["1"][1]) <= 1e-5


@pytest.mark.parametrize("pers", [0, 1])
def test_uniform_weight_kernel_instances(qs, monkeypatch, pers):
    """Two uniform instances of different density, gamma and length (1024 and
    2048 cells: one and two warps per line, four and two lines per 128-thread
    CTA) through the uniform-weight kernel, each line with its own instance's
    weight: bit for bit the per-cell-weight kernel, and each instance against
    its oracle."""
    base = synth.scaled(synth.SLAB_2D, dxi=0.05, k_list=[0.3, 0.9, 1.7, 2.6], profile="flattop", dt=1.5)
    insts = [synth.scaled(base, n_xi=1024, length=1024 * 0.05, gamma_b=20.0, species=[(-1.0, 1.0, 0.02)]),
             synth.scaled(base, n_xi=2048, length=2048 * 0.05, gamma_b=50.0, species=[(-1.0, 1.0, 0.05)])]
    out = {}
    for env in ("0", "1"):
        monkeypatch.setenv("QS_RES_NO_UNIFORM", env)
        s = qs.Solver(insts, prec="fp32")
        s.set_launch(**_res(32, 4, pers, 2))
        s.seed_noise(0, 1e-6)
        s.step(40)
        s.sync()
        out[env] = s.state_arrays()
        s.close()
    for a, b in zip(out["0"], out["1"]):
        for i in range(2):
            assert np.array_equal(a[i], b[i]), i
    nb, th = out["0"]
    for i, p in enumerate(insts):
        nb_o, th_o = oracle.seed_noise(p, 0, 1e-6, inst=i)
        oracle.sweep(p, nb_o, th_o, 0, 40)
        assert _log_err(nb[i], nb_o) <= FP32_LOG_TOL, i
        assert _log_err(th[i], th_o) <= FP32_LOG_TOL, i
