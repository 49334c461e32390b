"""C-ABI checks that need no GPU: the library loads, exports every symbol the
header declares, and rejects bad arguments on the host before touching CUDA."""
import ctypes
import os
import re

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def qs():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2607_24234_b300 as mod
    return mod


def test_exports_every_declared_symbol(qs):
    hdr = open(os.path.join(ROOT, "include", "qs.h")).read()
    names = sorted(set(re.findall(r"\b(qs_[a-z_0-9]+)\s*\(", hdr)))
    assert len(names) >= 15
    for n in names:
        assert hasattr(qs.lib, n), n
    assert set(qs.EXPORTS) <= set(names)


def _init(qs, problem, prec="fp32", n_inst=1, alloc=None):
    keep = []
    p = qs.make_params(problem, prec, keep)
    ctx = ctypes.c_void_p()
    st = qs.lib.qs_init(ctypes.byref(p), n_inst, None, alloc, None, ctypes.byref(ctx))
    return st, ctx


@pytest.mark.parametrize("field,value", [
    ("n_xi", 0), ("dxi", 0.0), ("dt", -1.0), ("gamma_b", 1.0), ("species", []),
    ("species", [(-1, 1, 0.01)] * 3), ("species", [(-1, 0.0, 0.01)]), ("species", [(-1, 1, -0.1)]),
    ("k_list", []), ("profile_gauss_sigma", 0.0),
])
def test_argument_errors_rejected_on_host(qs, field, value):
    p = synth.scaled(synth.SLAB_2D)
    if field == "profile_gauss_sigma":
        p.update(profile="gaussian", sigma_xi=value)
    else:
        p[field] = value
    if field == "species" and len(value) in (0, 3):
        # species counts outside 1..2: set the count by hand
        keep = []
        prm = qs.make_params(synth.SLAB_2D, "fp32", keep)
        prm.n_species = len(value)
        ctx = ctypes.c_void_p()
        st = qs.lib.qs_init(ctypes.byref(prm), 1, None, None, None, ctypes.byref(ctx))
    else:
        st, ctx = _init(qs, p)
    assert st == qs.QS_ERR_ARG
    assert ctx.value is None
    assert len(qs.lib.qs_last_error(None)) > 0


def test_other_host_errors(qs):
    keep = []
    p = qs.make_params(synth.SLAB_2D, "fp32", keep)
    ctx = ctypes.c_void_p()
    assert qs.lib.qs_init(ctypes.byref(p), 0, None, None, None, ctypes.byref(ctx)) == qs.QS_ERR_ARG
    assert qs.lib.qs_init(None, 1, None, None, None, ctypes.byref(ctx)) == qs.QS_ERR_ARG
    p.geom = 2   # finite-width real-space geometry is not served by this entry point
    assert qs.lib.qs_init(ctypes.byref(p), 1, None, None, None, ctypes.byref(ctx)) == qs.QS_ERR_UNSUPPORTED
    # held front without values
    q = qs.make_params(synth.scaled(synth.SLAB_2D, front="held"), "fp64", keep)
    assert qs.lib.qs_init(ctypes.byref(q), 1, None, None, None, ctypes.byref(ctx)) == qs.QS_ERR_ARG
    # per-instance parameters must share the k set
    a = synth.scaled(synth.SLAB_2D)
    b = synth.scaled(synth.SLAB_2D, k_list=[1.0, 2.0])
    per = (qs.Params * 2)(qs.make_params(a, "fp32", keep), qs.make_params(b, "fp32", keep))
    base = qs.make_params(a, "fp32", keep)
    assert qs.lib.qs_init(ctypes.byref(base), 2, per, None, None, ctypes.byref(ctx)) == qs.QS_ERR_ARG


def test_allocator_failure_reports_oom(qs):
    """A caller allocator that returns NULL yields QS_ERR_OOM (host-side
    failure injection: no device is touched)."""
    calls = []

    def _a(n, u):
        calls.append(int(n))
        return None

    def _f(ptr, u):
        pass

    al = qs.Allocator(qs.Allocator._fields_[0][1](_a), qs.Allocator._fields_[1][1](_f), None)
    st, ctx = _init(qs, synth.SLAB_2D, alloc=ctypes.byref(al))
    assert st == qs.QS_ERR_OOM
    assert calls and calls[0] == 512 * 64 * 16 + 256   # first request: the FP32 state and its 256-byte guard
    assert ctx.value is None


def test_null_context_calls(qs):
    v = ctypes.c_int64()
    assert qs.lib.qs_step(None, 1) == qs.QS_ERR_ARG
    assert qs.lib.qs_query(None, 0, 0, ctypes.byref(v)) == qs.QS_ERR_ARG
    assert qs.lib.qs_sync(None) == qs.QS_ERR_ARG
    qs.lib.qs_free(None)


@pytest.mark.parametrize("field,value", [
    ("dt", float("nan")), ("dt", float("inf")), ("dxi", float("nan")), ("gamma_b", float("nan")),
    ("gamma_b", float("inf")), ("species", [(float("nan"), 1.0, 0.01)]), ("species", [(-1.0, 1.0, float("inf"))]),
    ("k_list", [1.0, float("nan")]),
])
def test_nonfinite_parameters_rejected_by_both_entry_points(qs, field, value):
    """qs_init and the allocation-free qs_sweep_noalloc share one check of the
    problem statement: a non-finite parameter is an argument error, returned
    on the host before any CUDA call."""
    p = synth.scaled(synth.SLAB_2D, **{field: value})
    st, ctx = _init(qs, p)
    assert st == qs.QS_ERR_ARG and ctx.value is None
    keep = []
    prm = qs.make_params(p, "fp32", keep)
    dummy = ctypes.c_void_p(0x1000)   # never dereferenced: the call returns first
    ex = ctypes.cast(dummy, ctypes.POINTER(ctypes.c_int))
    assert qs.lib.qs_sweep_noalloc(ctypes.byref(prm), dummy, None, ex, 0, 1, None, None) == qs.QS_ERR_ARG
    prm.geom = 2
    assert qs.lib.qs_sweep_noalloc(ctypes.byref(prm), dummy, None, ex, 0, 1, None, None) == qs.QS_ERR_UNSUPPORTED


def test_growth_bound_and_renormalisation_interval(qs):
    """qs_growth_bound (host only): the benchmark beam keeps the resident
    sweep's 16-step renormalisation interval, every instance of the batched
    workload gets an interval, and an extreme problem is refused (0)."""
    g, ev = qs.growth_bound(synth.BEAM_3D)
    assert 0.0 < g < 0.1 and ev == 16
    evs = [qs.growth_bound(p)[1] for p in synth.batch_instances(512, param_seed=0)]
    assert min(evs) >= 4 and max(evs) == 16
    assert sorted(evs)[:3] == [8, 8, 16]      # the two densest, slowest beams check every 8 steps
    # the interval shrinks as the bound grows, down to refusal
    prev = 16
    for dens, dt in ((1.0, 20.0), (10.0, 100.0), (100.0, 1000.0)):
        extreme = synth.scaled(synth.SLAB_2D, species=[(-1.0, 1.0, dens)], gamma_b=1.1, dt=dt, n_xi=4000, dxi=0.25,
                               length=1000.0)
        g, ev = qs.growth_bound(extreme)
        assert ev <= prev
        prev = ev
    assert ev == 0 and g > 20.0
    with pytest.raises(qs.QSError):
        qs.growth_bound(synth.scaled(synth.SLAB_2D, dt=float("nan")))


@pytest.mark.parametrize("species,gamma,dt,L", [
    ([(-1.0, 1.0, 0.1)], 10.0, 2.0, 20.0),
    ([(-1.0, 1.0, 0.3)], 2.0, 4.0, 10.0),
    ([(-1.0, 1.0, 0.05), (1.0, 1.0, 0.05)], 3.0, 2.0, 15.0),
])
def test_growth_bound_bounds_the_oracle(qs, species, gamma, dt, L):
    """The bound is an upper bound of the scheme's growth: from random states
    (n_b and Theta both non-zero), the FP64 oracle's max norm over n_b and
    Theta after k steps never exceeds e^(k g) times the one-time factor
    sqrt(2 max(a, b) / min(a, b)) times the initial one."""
    import math
    import oracle
    n_xi, D = int(round(L / 0.05)), 0.05
    p = synth.scaled(synth.SLAB_2D, species=species, gamma_b=gamma, dt=dt, n_xi=n_xi, dxi=D, length=n_xi * D,
                     k_list=[0.0, 0.7, 2.0, 6.0])
    g, ev = qs.growth_bound(p)
    qm = max(abs(q / m) for q, m, _ in species)
    a = dt * qm * (1 / gamma + 1 / gamma ** 3) * sum(abs(q) for q, _, _ in species) * (2 + n_xi * D)
    b = dt * max(d for _, _, d in species)
    lc = 0.5 * abs(math.log(a / b)) + 0.5 * math.log(2.0)
    rng = np.random.default_rng(3)
    for trial in range(3):
        nb = rng.standard_normal((4, len(species), n_xi)) + 1j * rng.standard_normal((4, len(species), n_xi))
        th = (rng.standard_normal(nb.shape) + 1j * rng.standard_normal(nb.shape)) * 10.0 ** (trial - 1)
        m0 = max(np.max(np.abs(nb)), np.max(np.abs(th)))
        for k in range(1, 13):
            oracle.sweep(p, nb, th, k, 1)
            mk = max(np.max(np.abs(nb)), np.max(np.abs(th)))
            assert math.log(mk / m0) <= k * g + lc + 1e-9, (trial, k)


def test_bounds_checked_build(qs):
    """The bounds-checked variant (libqs_checked.so, -DQS_CHECK_BOUNDS) is
    built beside the ordinary one, reports itself through qs_build_flags and
    exports every symbol the header declares."""
    hdr = open(os.path.join(ROOT, "include", "qs.h")).read()
    names = sorted(set(re.findall(r"\b(qs_[a-z_0-9]+)\s*\(", hdr)))
    path = os.path.join(ROOT, "paper_2607_24234_b300", "libqs_checked.so")
    L = ctypes.CDLL(path)
    assert L.qs_build_flags() == qs.BUILD_CHECK_BOUNDS
    assert qs.lib.qs_build_flags() == 0
    for n in names:
        assert hasattr(L, n), n


def test_stale_library_is_refused(qs, tmp_path):
    """The binding loads a library only if the hash of its sources, written
    beside it by the build, matches the current sources: a library built from
    other sources is refused at import, not run."""
    import shutil
    import subprocess
    import sys
    lib = os.path.join(ROOT, "paper_2607_24234_b300", "libqs.so")
    assert open(lib + ".srchash").read().strip() == qs._source_hash()
    stale = tmp_path / "libqs.so"
    shutil.copy(lib, stale)
    (tmp_path / "libqs.so.srchash").write_text("0" * 64 + "\n")
    r = subprocess.run([sys.executable, "-c", "import paper_2607_24234_b300"], cwd=ROOT, capture_output=True,
                       text=True, env=dict(os.environ, QS_LIBRARY=str(stale)))
    assert r.returncode != 0 and "not built from the current sources" in r.stderr
