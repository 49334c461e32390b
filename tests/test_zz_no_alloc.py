"""qs_sweep_noalloc: the allocation-free entry point, for callers that must not
allocate device memory while they step the solver (their framework owns every
device buffer, or an allocation there could synchronise the device or fail).

The caller keeps the state in its own buffers; the test builds them from a
checkpoint of the regular path, advances them with two calls in a row through
the C ABI and compares the result with qs_step on the same problem, within
the tolerances of the other GPU tests.  This file is collected last.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2607_24234_b300 as m
    return m


def _decode(prec, st, th, ex, n_xi, NS, Mp, M):
    """Caller buffers -> complex n_b, Theta as [mode][species][xi]."""
    if prec == "fp32":
        a = st.view(np.float32).reshape(n_xi, NS, Mp, 4).astype(np.float64)
        W = (ex.view(np.int32).reshape(-1, Mp) >> 8).astype(np.int64)
        a = np.ldexp(a, W[np.arange(n_xi) // 32][:, None, :, None])
        nb, tt = a[..., 0] + 1j * a[..., 1], a[..., 2] + 1j * a[..., 3]
    else:
        a = st.view(np.float64).reshape(n_xi, NS, Mp, 2)
        b = th.view(np.float64).reshape(n_xi, NS, Mp, 2)
        nb, tt = a[..., 0] + 1j * a[..., 1], b[..., 0] + 1j * b[..., 1]
    return (np.transpose(nb[:, :, :M], (2, 1, 0)), np.transpose(tt[:, :, :M], (2, 1, 0)))


@pytest.mark.parametrize("prec,species", [
    ("fp32", [(-1.0, 1.0, 0.01)]),
    ("fp64", [(-1.0, 1.0, 0.03), (1.0, 1.0, 0.03)]),
])
def test_noalloc_matches_regular_path_two_calls(qs, prec, species):
    import torch
    p = synth.scaled(synth.BEAM_3D, nkx=40, nky=40, kmax=6.0, n_xi=300, dxi=0.05, length=15.0,
                     species=species, gamma_b=200.0)
    n1, n2 = 7, 11
    stream = torch.cuda.current_stream()
    ref = qs.Solver(p, prec=prec)
    ref.seed_noise(9, 1e-6)
    ck = ref.checkpoint()
    ref.step(n1)
    ref.step(n2)
    ref.sync()
    nb_ref, th_ref = ref.state_arrays()
    M, Mp, NS, n_xi = ref.n_modes, ref.Mp, len(species), p["n_xi"]
    ref.close()

    # the caller's own buffers, filled from the checkpoint (after its header)
    body = ck[64:]
    esz = 16
    nst = n_xi * NS * Mp * esz
    st = torch.from_numpy(body[:nst].copy()).cuda()
    th = ex = None
    if prec == "fp64":
        th = torch.from_numpy(body[nst:2 * nst].copy()).cuda()
    else:
        ex = torch.from_numpy(body[nst:].copy()).cuda()
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    keep = []
    prm = qs.make_params(p, prec, keep)

    def call(step0, n):
        return qs.lib.qs_sweep_noalloc(
            ctypes.byref(prm), ctypes.c_void_p(st.data_ptr()),
            ctypes.c_void_p(th.data_ptr()) if th is not None else None,
            ctypes.cast(ctypes.c_void_p(ex.data_ptr()), ctypes.POINTER(ctypes.c_int)) if ex is not None else None,
            step0, n, ctypes.cast(ctypes.c_void_p(status.data_ptr()), ctypes.POINTER(ctypes.c_int)),
            ctypes.c_void_p(stream.cuda_stream))

    assert call(0, n1) == qs.QS_OK
    assert call(n1, n2) == qs.QS_OK
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    nb, tt = _decode(prec, st.cpu().numpy(), th.cpu().numpy() if th is not None else None,
                     ex.cpu().numpy() if ex is not None else None, n_xi, NS, Mp, M)
    if prec == "fp64":
        for a, b in ((nb, nb_ref), (tt, th_ref)):
            rel = np.max(np.abs(a - b)) / np.max(np.abs(b))
            assert rel <= 1e-9
    else:
        for a, b in ((nb, nb_ref), (tt, th_ref)):
            m = np.abs(b) >= 1e-3 * np.max(np.abs(b).reshape(M, -1), axis=1)[:, None, None]
            assert np.max(np.abs(np.log(np.abs(a[m])) - np.log(np.abs(b[m])))) <= 1e-3


def test_noalloc_rejects_sizes_beyond_its_scratch(qs):
    import torch
    keep = []
    big = synth.scaled(synth.BEAM_3D, nkx=1024, nky=1024, n_xi=64)    # ~820k modes
    prm = qs.make_params(big, "fp32", keep)
    buf = torch.zeros(16, dtype=torch.uint8, device="cuda")
    exb = torch.zeros(4, dtype=torch.int32, device="cuda")
    st = qs.lib.qs_sweep_noalloc(ctypes.byref(prm), ctypes.c_void_p(buf.data_ptr()), None,
                                 ctypes.cast(ctypes.c_void_p(exb.data_ptr()), ctypes.POINTER(ctypes.c_int)),
                                 0, 1, None, None)
    assert st == qs.QS_ERR_ARG
    held = qs.make_params(synth.scaled(synth.SLAB_2D, front="held"), "fp32", keep)
    st = qs.lib.qs_sweep_noalloc(ctypes.byref(held), ctypes.c_void_p(buf.data_ptr()), None,
                                 ctypes.cast(ctypes.c_void_p(exb.data_ptr()), ctypes.POINTER(ctypes.c_int)),
                                 0, 1, None, None)
    assert st == qs.QS_ERR_UNSUPPORTED


# the refused call enqueues nothing, so torch reports the captured graph as empty
@pytest.mark.filterwarnings("ignore:The CUDA Graph is empty:UserWarning")
def test_noalloc_refuses_a_capturing_stream(qs):
    """The tables come from pageable host memory, so a call made while its
    stream is being captured into a CUDA graph is refused with nothing
    enqueued (a captured copy would read host memory that is gone when the
    graph runs); the same call outside capture works."""
    import torch
    p = synth.scaled(synth.BEAM_3D, nkx=16, nky=16, kmax=6.0, n_xi=64, dxi=0.05, length=3.2)
    keep = []
    prm = qs.make_params(p, "fp32", keep)
    ref = qs.Solver(p, prec="fp32")
    ref.seed_noise(1, 1e-6)
    ck = ref.checkpoint()
    Mp = ref.Mp
    ref.close()
    body = ck[64:]
    nst = p["n_xi"] * Mp * 16
    st = torch.from_numpy(body[:nst].copy()).cuda()
    ex = torch.from_numpy(body[nst:].copy()).cuda()
    exp_ = ctypes.cast(ctypes.c_void_p(ex.data_ptr()), ctypes.POINTER(ctypes.c_int))
    side = torch.cuda.Stream()

    def call():
        return qs.lib.qs_sweep_noalloc(ctypes.byref(prm), ctypes.c_void_p(st.data_ptr()), None, exp_, 0, 2,
                                       None, ctypes.c_void_p(side.cuda_stream))

    assert call() == qs.QS_OK          # the first call on the device sets up the scratch address
    side.synchronize()
    before = st.clone()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        rc = call()
    assert rc == qs.QS_ERR_UNSUPPORTED
    torch.cuda.synchronize()
    assert torch.equal(st, before)     # nothing was enqueued
    assert call() == qs.QS_OK
    side.synchronize()
