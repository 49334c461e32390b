"""Runs under the bounds-checked library (QS_LIBRARY=libqs_checked.so), in a
process of its own: every sweep variant on small cases, each checked against
the FP64 oracle and required to finish without a bounds report; then the
bounds hook (the checker told that the last state rows are missing) must
produce QS_ERR_BOUNDS.  Prints one line per case and 'ALL OK' at the end."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))

import torch  # noqa: E402

import paper_2607_24234_b300 as qs  # noqa: E402
import synth  # noqa: E402
from test_gpu_parity import FP32_LOG_TOL, _log_err, _run_oracle  # noqa: E402


def case(name, p, prec, launch, steps=9, rec=0):
    s = qs.Solver(p, prec=prec)
    if launch:
        s.set_launch(**launch)
    s.seed_noise(4, 1e-6)
    if rec:
        s.record(rec, 3, (steps + 2) // 3)
    s.step(steps)
    s.sync()
    if rec:
        s.record(0, 1, 0)
    s.diag(qs.REC_MAG)
    nb, th = s.state_arrays()
    s.close()
    nb_o, th_o = _run_oracle(p, steps, seed=("noise", 4, 1e-6))
    if prec == "fp64":
        err = np.max(np.abs(nb - nb_o)) / np.max(np.abs(nb_o))
        assert err <= 1e-9, (name, err)
    else:
        assert _log_err(nb, nb_o) <= FP32_LOG_TOL and _log_err(th, th_o) <= FP32_LOG_TOL, name
    print("ok", name, flush=True)


def main():
    assert qs.lib.qs_build_flags() == qs.BUILD_CHECK_BOUNDS, "not the bounds-checked build"
    torch.cuda.set_device(0)
    p = synth.scaled(synth.BEAM_3D, nkx=20, nky=20, kmax=5.0, n_xi=300, dxi=0.05, length=15.0, gamma_b=50.0)
    p2 = synth.scaled(p, species=[(-1.0, 1.0, 0.02), (1.0, 1.0, 0.02)])
    held = synth.scaled(synth.SLAB_2D, n_xi=130, dxi=0.05, length=6.5, k_list=[0.5, 2.0, 4.0], front="held")
    for prec in ("fp32", "fp64"):
        case(f"registers-{prec}", p, prec, dict(warps_per_cta=2, prefetch=4 if prec == "fp32" else 2, persistent=1,
                                                ctas_per_sm=4, variant=0))
        case(f"tma-{prec}", p2, prec, dict(warps_per_cta=1, prefetch=8 if prec == "fp32" else 4, persistent=0,
                                           ctas_per_sm=8, variant=1))
        case(f"record-{prec}", p, prec, None, rec=qs.REC_MAG | qs.REC_NP | qs.REC_MODEMAX)
    case("scan-fp64", synth.scaled(synth.SLAB_2D, n_xi=200, dxi=0.05, length=10.0, k_list=[1.0, 3.0]), "fp64",
         dict(warps_per_cta=1, prefetch=8, persistent=0, ctas_per_sm=8, variant=2, scan_cells=8))
    for V, w, sc in ((32, 2, 8), (32, 1, 1), (16, 4, 8), (8, 2, 8)):
        case(f"resident-V{V}-w{w}-t{sc}", p, "fp32", dict(warps_per_cta=w, prefetch=V, persistent=1, ctas_per_sm=2,
                                                          variant=3, scan_cells=sc))
    case("resident-2sp-V16", p2, "fp32", dict(warps_per_cta=4, prefetch=16, persistent=0, ctas_per_sm=1, variant=3))
    case("resident-modemax", p, "fp32", dict(warps_per_cta=2, prefetch=32, persistent=0, ctas_per_sm=1, variant=3),
         rec=qs.REC_MODEMAX)
    s = qs.Solver(held, prec="fp32", held=np.full((3, 4), 1e-7))
    s.set_launch(warps_per_cta=2, prefetch=16, persistent=0, ctas_per_sm=1, variant=3)
    s.seed_noise(1, 1e-6)
    s.step(5)
    s.sync()
    s.close()
    print("ok held-front-resident", flush=True)
    g = qs.Solver(synth.scaled(synth.SLAB_2D, n_xi=300, dxi=0.05, length=15.0, k_list=[0.5, 2.0]), prec="fp32")
    g.seed_noise(2, 1e-6)
    g.step_green(7)
    g.step_green(5)
    g.sync()
    g.close()
    print("ok green", flush=True)
    # detection: the checker is told the last 10 state rows are missing
    s = qs.Solver(p, prec="fp32")
    s.seed_noise(4, 1e-6)
    s.debug_bounds(10)
    s.step(2)
    try:
        s.sync()
        raise AssertionError("no bounds report")
    except qs.QSError as e:
        assert e.status == qs.QS_ERR_BOUNDS, e
        print("ok detected:", str(e), flush=True)
    s.close()
    print("ALL OK", flush=True)


if __name__ == "__main__":
    main()
