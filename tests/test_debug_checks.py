"""Failure detection of the debug aids, on the GPU without a fault:

- the guard (canary) after every context buffer: a host-side overwrite of one
  guard byte (inside the allocation) is reported by the next qs_sync;
- the bounds-checked build: every sweep variant runs clean against the
  oracle, and the bounds hook (the checker is told that state rows are
  missing; the memory is there) is reported as QS_ERR_BOUNDS.
"""
import os
import subprocess
import sys

import pytest

import synth

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def qs():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2607_24234_b300 as m
    return m


def test_canary_overwrite_is_reported(qs):
    import ctypes
    p = synth.scaled(synth.SLAB_2D, n_xi=100, dxi=0.05, length=5.0, k_list=[1.0, 2.0])
    s = qs.Solver(p, prec="fp32")
    s.seed_noise(1, 1e-6)
    s.step(3)
    s.sync()                                   # clean guards
    qs.lib.qs_debug_canary.argtypes = [ctypes.c_void_p, ctypes.c_int]
    assert qs.lib.qs_debug_canary(s.ctx, 0) == qs.QS_OK
    with pytest.raises(qs.QSError) as e:
        s.sync()
    assert e.value.status == qs.QS_ERR_BOUNDS and "guard" in str(e.value)
    s.close()


def test_bounds_checked_build_runs_clean_and_detects():
    lib = os.path.join(ROOT, "paper_2607_24234_b300", "libqs_checked.so")
    env = dict(os.environ, QS_LIBRARY=lib)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "checked_build_cases.py")], env=env,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    assert "ALL OK" in r.stdout and "ok detected" in r.stdout
