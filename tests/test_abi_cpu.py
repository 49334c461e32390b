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
    assert calls and calls[0] == 512 * 64 * 16   # first request: the FP32 state
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
