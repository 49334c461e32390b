"""GPU checks of the learned surrogate.

- Forward outputs and gradients of the BF16 tensor-core kernels against the
  FP64 CPU backprop (itself pinned by finite differences) on identical
  BF16-rounded weights and inputs: forward rel. L2 <= 1e-2, gradients
  rel. L2 <= 2e-2 per tensor.
- Training samples drawn on the GPU against the CPU restatement of the
  targets on the oracle's own fields.
- A trained ensemble on held-out parameter sets: envelope error, class
  accuracy, the solver fallback, and the time it saves over the solver.
"""
import ctypes
import math
import time

import numpy as np
import pytest

import oracle
import synth
from oracle import mlp as omlp
from oracle import surdata

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_2607_24234_b300 as qs
    from paper_2607_24234_b300 import surrogate
    return qs, surrogate


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.mark.parametrize("no_fused,no_tc,n", [("0", "0", 1000), ("1", "0", 1000), ("0", "0", 1003), ("0", "1", 1000)])
def test_forward_and_gradients_match_fp64(sg, monkeypatch, no_fused, no_tc, n):
    """Every training path: the fused forward (loss and output-layer backward
    in its epilogue, gelu' stored for the backward GEMMs), the layer-by-
    layer tcgen05 path, and the mma.sync kernels (QS_MLP_NO_TCGEN05=1);
    n = 1003 is not a multiple of 8 (no tensor-core weight gradient: the
    transposed operands go through the mma.sync kernel)."""
    import torch
    qs, sur = sg
    monkeypatch.setenv("QS_MLP_NO_FUSED", no_fused)
    monkeypatch.setenv("QS_MLP_NO_TCGEN05", no_tc)
    rng = np.random.default_rng(0)
    X = (rng.standard_normal((n, 7)) * np.array([1.0, 2.0, 50.0, 30.0, 500.0, 2.0, 1.5])
         + np.array([-4.0, 6.0, 100.0, 40.0, 900.0, 3.0, 0.0])).astype(np.float32)
    Y = np.stack([10 * rng.standard_normal(n) + 20, (rng.random(n) > 0.4)], axis=1).astype(np.float32)
    Xt, Yt = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    m = sur.MLP(width=256, depth=3, ensemble=2, max_batch=1024, seed=1)
    m.set_norm(Xt, Yt)
    flat = m.params(0)
    for W, b in m.layers(flat):
        b[:] = 0.1 * rng.standard_normal(b.shape)
    m.set_params(flat, 0)
    m.set_params(flat, 1)
    m.train_step(Xt, Yt, 0.0, update=False)
    g = m.grads(0)
    mean, inv_std, ymean, ystd = m.norm()
    xs = np.zeros((n, 16))
    xs[:, :7] = omlp.bf16((X - mean[:7].astype(np.float32)) * inv_std[:7].astype(np.float32))
    layers = [(omlp.bf16(W), b.astype(np.float64)) for W, b in m.layers(flat)]
    _, grads, out = omlp.loss_and_grads(layers, xs, Y.astype(np.float64), ymean, ystd)
    for l, ((gW, gb), (oW, ob)) in enumerate(zip(m.layers(g), grads)):
        assert _rel(gW, oW) <= 2e-2, ("W", l, _rel(gW, oW))
        assert _rel(gb, ob) <= 2e-2, ("b", l, _rel(gb, ob))
    mu, var, mask = m.infer(Xt)
    mu = mu.cpu().numpy()
    assert _rel(mu[:, 0], out[:, 0] * ystd + ymean) <= 1e-2
    assert _rel(mu[:, 1], out[:, 1]) <= 1e-2
    assert float(var.max()) <= 1e-6 * max(1.0, float(np.max(np.abs(mu)))) ** 2
    m.close()


def test_fused_training_split_last_round(sg, monkeypatch):
    """16,384 rows x 4 members are 512 (tile, member) items; on 148 SMs the
    last round's 68 items are split into 64-row halves by the fused forward
    and the input-gradient kernel.  The loss and every member's gradients
    equal those of the unsplit launches (QS_MLP_NO_SPLIT=1) up to the order
    of the atomic sums.  A 64-row half dropped or counted twice would move
    them by about 64/16,384 = 4e-3, far above the 1e-5 bound."""
    import torch
    qs, sur = sg
    n = 16384
    rng = np.random.default_rng(3)
    X = (rng.standard_normal((n, 7)) * np.array([1.0, 2.0, 50.0, 30.0, 500.0, 2.0, 1.5])
         + np.array([-4.0, 6.0, 100.0, 40.0, 900.0, 3.0, 0.0])).astype(np.float32)
    Y = np.stack([10 * rng.standard_normal(n) + 20, (rng.random(n) > 0.4)], axis=1).astype(np.float32)
    Xt, Yt = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    out = {}
    for env in ("0", "1"):
        monkeypatch.setenv("QS_MLP_NO_SPLIT", env)
        m = sur.MLP(width=256, depth=3, ensemble=4, max_batch=n, seed=1)
        m.set_norm(Xt, Yt)
        loss = m.train_step(Xt, Yt, 0.0, update=False, want_loss=True)
        out[env] = (loss, [m.grads(e) for e in range(4)])
        m.close()
    assert abs(out["0"][0] - out["1"][0]) <= 1e-5 * abs(out["1"][0])
    for e in range(4):
        assert _rel(out["0"][1][e], out["1"][1][e]) <= 1e-5, e
    assert np.isfinite(out["0"][0]) and out["0"][0] > 0


@pytest.mark.parametrize("width,depth", [(256, 3), (48, 2)])
def test_adam_writes_the_transposed_weights(sg, monkeypatch, width, depth):
    """Adam writes the bf16 copies W^T that the next step's input-gradient
    kernels read, in 32 x 32 tiles of each weight matrix.  Three updating
    steps, then the loss and the gradients of a fourth, against the same run
    with the copies made by a separate pass after the update
    (QS_MLP_WT_PASS=1).  The values written are the same; the runs differ
    only in the order of their atomic sums.  A wrong or stale W^T would give
    wrong input gradients from the second step on.  Width 48 leaves tiles
    16 columns wide at each matrix's edge, and the 2-row output layer fills
    two rows of its tiles."""
    import torch
    qs, sur = sg
    n = 4096
    rng = np.random.default_rng(5)
    X = (rng.standard_normal((n, 7)) * 3).astype(np.float32)
    Y = np.stack([10 * rng.standard_normal(n) + 20, (rng.random(n) > 0.4)], axis=1).astype(np.float32)
    Xt, Yt = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    out = {}
    for env in ("0", "1"):
        monkeypatch.setenv("QS_MLP_WT_PASS", env)
        m = sur.MLP(width=width, depth=depth, ensemble=2, max_batch=n, seed=2)
        m.set_norm(Xt, Yt)
        for _ in range(3):
            m.train_step(Xt, Yt, 3e-3)
        loss = m.train_step(Xt, Yt, 0.0, update=False, want_loss=True)
        out[env] = (loss, [m.grads(e) for e in range(2)])
        m.close()
    assert abs(out["0"][0] - out["1"][0]) <= 1e-4 * abs(out["1"][0])
    for e in range(2):
        assert _rel(out["0"][1][e], out["1"][1][e]) <= 1e-3, e


def test_training_samples_match_oracle_targets(sg):
    import torch
    qs, sur = sg
    insts = synth.batch_instances(3, param_seed=7, base=synth.scaled(synth.BATCH_BASE, nkx=12, nky=12),
                                  dxi=0.1)
    steps, amp, n = 60, 1e-6, 3000
    s = qs.Solver(insts, prec="fp64")
    s.seed_noise(0, amp)
    s.step(steps)
    snap = s.diag(qs.REC_MAG, host=False)
    X = torch.empty((n, 7), dtype=torch.float32, device="cuda")
    Y = torch.empty((n, 2), dtype=torch.float32, device="cuda")
    st = qs.lib.qs_sur_points(s.ctx, ctypes.c_void_p(snap.data_ptr()), snap.numel() * 8, amp, n, 5,
                              ctypes.c_void_p(X.data_ptr()), ctypes.c_void_p(Y.data_ptr()))
    assert st == 0
    X, Y = X.cpu().numpy(), Y.cpu().numpy()
    md = oracle.modes(insts[0])
    ang = np.arctan2(md["ky"], md["kx"]).astype(np.float32)
    kab = np.sqrt(md["kx"] ** 2 + md["ky"] ** 2).astype(np.float32)
    mags = []
    for i, p in enumerate(insts):
        nb, th = oracle.seed_noise(p, 0, amp, inst=i)
        oracle.sweep(p, nb, th, 0, steps)
        mags.append(oracle.fields(p, nb)["mag"])
    feats = np.array([[np.float32(np.log(p["species"][0][2])), np.float32(np.log(p["gamma_b"]))]
                      for p in insts])
    bad0, bad1 = 0, 0
    for r in range(n):
        i = int(np.argmin(np.abs(feats[:, 0] - X[r, 0]) + np.abs(feats[:, 1] - X[r, 1])))
        p = insts[i]
        j = int(round(X[r, 3] / p["dxi"] - 0.5))
        mo = int(np.argmin(np.abs(kab - X[r, 5]) + np.abs(ang - X[r, 6])))
        y0, y1 = surdata.targets(mags[i][:, mo, :], p["dxi"], j, amp)
        bad0 += abs(y0 - Y[r, 0]) > 1e-4 * max(1.0, abs(y0))
        bad1 += y1 != Y[r, 1]
    assert bad0 == 0
    assert bad1 <= n // 200
    s.close()


@pytest.mark.slow
def test_surrogate_learns_and_screens_heldout(sg):
    """Train on solver sweeps of 16 parameter sets, evaluate on 8 held-out
    sets (parameter seed 1): the ensemble answers screening queries far
    faster than the solver produces them, at a stated error; flagged queries
    fall back to the solver."""
    import torch
    qs, sur = sg
    base = synth.scaled(synth.BATCH_BASE, nkx=32, nky=32)
    snaps = [200, 400, 600, 800, 1000]
    tr = synth.batch_instances(16, param_seed=0, base=base, dxi=0.05)
    ho = synth.batch_instances(8, param_seed=1, base=base, dxi=0.05)
    Xtr, Ytr, _ = sur.generate(tr, snaps, 1 << 16, seed=1)
    Xho, Yho, solver_s = sur.generate(ho, snaps, 1 << 14, seed=2, noise_seed=1)
    assert torch.isfinite(Xtr).all() and torch.isfinite(Ytr).all()
    m, losses = sur.train(Xtr, Ytr, epochs=12, batch=8192, lr=2e-3, ensemble=4, seed=3)
    assert losses[-1] < 0.5 * losses[0]
    res = sur.evaluate(m, Xho, Yho)
    mu, var, _ = m.infer(Xho)                 # warm
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mu, var, _ = m.infer(Xho)
    torch.cuda.synchronize()
    infer_s = time.perf_counter() - t0
    thr = float(torch.quantile(var[:, 0], 0.9))
    _, _, mask = m.infer(Xho, thr)
    flagged = float(mask.float().mean())
    print({"heldout": res, "flagged_at_p90_var": flagged, "solver_s": solver_s, "infer_s": infer_s})
    assert res["rmse"] < 0.35 * res["target_std"]
    assert res["accuracy"] > 0.8
    assert 0.05 < flagged < 0.2
    assert infer_s < 0.1 * solver_s          # screening gain over running the solver
    assert math.isfinite(res["rmse"])
    m.close()


def test_native_training_entry_points(sg):
    """qs_sur_train / qs_sur_infer: the whole training loop behind the C ABI
    (host-drawn shuffles, cosine learning rate) reaches the same quality
    bars on held-out parameter sets; the fallback mask follows the
    threshold."""
    import torch
    qs, sur = sg
    base = synth.scaled(synth.BATCH_BASE, nkx=32, nky=32)
    snaps = [200, 400, 600, 800, 1000]
    tr = synth.batch_instances(16, param_seed=0, base=base, dxi=0.05)
    ho = synth.batch_instances(8, param_seed=1, base=base, dxi=0.05)
    Xtr, Ytr, _ = sur.generate(tr, snaps, 1 << 16, seed=1)
    Xho, Yho, _ = sur.generate(ho, snaps, 1 << 14, seed=2, noise_seed=1)
    m = sur.SurModel(Xtr, Ytr, epochs=12, batch=8192, lr=2e-3, ensemble=4, seed=3)
    losses = m.losses()
    assert len(losses) == 12 and losses[-1] < 0.5 * losses[0]
    mu, var, mask = m.infer(Xho)
    err = (mu[:, 0] - Yho[:, 0])
    rmse = float(torch.sqrt(torch.mean(err * err)))
    acc = float(((mu[:, 1] > 0).float() == Yho[:, 1]).float().mean())
    assert rmse < 0.35 * float(Yho[:, 0].std()) and acc > 0.8
    assert int(mask.sum()) == 0                       # default threshold: no fallback
    m.set_threshold(float(torch.quantile(var[:, 0], 0.9)))
    _, _, mask = m.infer(Xho)
    frac = float(mask.float().mean())
    assert 0.05 < frac < 0.15
    m.close()


def test_screen_answers_flagged_queries_with_the_solver(sg):
    """qs_sur_screen: the ensemble answers every query; the rows above the
    variance threshold are answered by solver runs of their parameter sets.
    Unflagged rows equal qs_sur_infer's outputs bitwise; flagged rows equal
    the labels the solver wrote for the same queries (same noise) and an
    independent FP64 oracle run of the same set, at the FP32 bar (1e-3 in the
    log envelope; the class may differ on a knife-edge row or two)."""
    import torch
    qs, sur = sg
    base = synth.scaled(synth.BATCH_BASE, nkx=12, nky=12)
    insts = synth.batch_instances(4, param_seed=7, base=base, dxi=0.1)
    snaps, amp = [20, 40], 1e-6
    Xtr, Ytr, _ = sur.generate(insts, snaps, 4096, seed=1)
    Xq, Yq, _ = sur.generate(insts, snaps, 1024, seed=2, noise_seed=3)
    m = sur.SurModel(Xtr, Ytr, epochs=2, batch=2048, ensemble=2, seed=3)
    _, var, _ = m.infer(Xq)
    m.set_threshold(float(torch.quantile(var[:, 0], 0.7)))
    mu, var, mask0 = m.infer(Xq)
    y, v, mask, ns = m.screen(insts, Xq, noise_seed=3, amplitude=amp)
    torch.cuda.synchronize()
    mask = mask.bool()
    assert torch.equal(mask, mask0.bool())
    assert ns == int(mask.sum()) and 0.2 * len(mask) < ns < 0.4 * len(mask)
    assert torch.equal(y[~mask], mu[~mask]) and torch.equal(v[~mask], var[~mask])
    assert bool((v[mask] == 0).all())
    yf, Yf = y[mask].cpu().numpy(), Yq[mask].cpu().numpy()
    assert np.max(np.abs(yf[:, 0] - Yf[:, 0])) <= 1e-3
    assert np.sum((yf[:, 1] > 0) != (Yf[:, 1] > 0.5)) <= max(1, len(yf) // 100)
    # independent: the FP64 oracle's fields for the flagged rows
    Xf = Xq[mask].cpu().numpy()
    md = oracle.modes(insts[0])
    ang = np.arctan2(md["ky"], md["kx"]).astype(np.float32)
    kab = np.sqrt(md["kx"] ** 2 + md["ky"] ** 2).astype(np.float32)
    feats = np.array([[np.float32(np.log(p["species"][0][2])), np.float32(np.log(p["gamma_b"]))] for p in insts])
    mags = {}
    for i, p in enumerate(insts):
        nb, th = oracle.seed_noise(p, 3, amp, inst=i)
        done = 0
        for stp in snaps:
            oracle.sweep(p, nb, th, done, stp - done)
            done = stp
            mags[(i, stp)] = oracle.fields(p, nb)["mag"]
    bad0 = bad1 = 0
    for r in range(len(Xf)):
        i = int(np.argmin(np.abs(feats[:, 0] - Xf[r, 0]) + np.abs(feats[:, 1] - Xf[r, 1])))
        p = insts[i]
        stp = int(round(Xf[r, 4] / p["dt"]))
        j = int(round(Xf[r, 3] / p["dxi"] - 0.5))
        mo = int(np.argmin(np.abs(kab - Xf[r, 5]) + np.abs(ang - Xf[r, 6])))
        y0, y1 = surdata.targets(mags[(i, stp)][:, mo, :], p["dxi"], j, amp)
        bad0 += abs(y0 - yf[r, 0]) > 1e-3
        bad1 += (yf[r, 1] > 0) != (y1 > 0.5)
    assert bad0 == 0
    assert bad1 <= max(1, len(Xf) // 100)
    m.close()


def test_fused_inference_matches_layer_path_and_fp64(sg, monkeypatch):
    """The fused ensemble inference (one launch; every member's layers on
    chip, outputs and ensemble statistics in the last epilogue) against the
    layer-by-layer path and the FP64 forward of the CPU oracle on the same
    BF16-rounded weights and inputs, on a ragged row count: mean within
    rel. L2 1e-3 of the layer path and 1e-2 of FP64, variance within 2e-2
    of the layer path, and the same fallback mask away from the threshold."""
    import torch
    qs, sur = sg
    rng = np.random.default_rng(4)
    n = 5003                                   # 39 full 128-row tiles and a ragged one
    X = (rng.standard_normal((n, 7)) * np.array([1.0, 2.0, 50.0, 30.0, 500.0, 2.0, 1.5])
         + np.array([-4.0, 6.0, 100.0, 40.0, 900.0, 3.0, 0.0])).astype(np.float32)
    Y = np.stack([10 * rng.standard_normal(n) + 20, (rng.random(n) > 0.4)], axis=1).astype(np.float32)
    Xt, Yt = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    models = {}
    for tag, env in (("fused", "0"), ("layers", "1")):
        monkeypatch.setenv("QS_MLP_NO_FUSED", env)
        m = sur.MLP(width=256, depth=3, ensemble=4, max_batch=2048, seed=9)
        m.set_norm(Xt, Yt)
        models[tag] = m
    flats = []
    for e in range(4):
        flat = models["fused"].params(e)
        for W, b in models["fused"].layers(flat):
            b[:] = 0.2 * rng.standard_normal(b.shape)
        flats.append(flat)
        for m in models.values():
            m.set_params(flat, e)
    thr = 0.05
    res = {tag: [t.cpu().numpy() for t in m.infer(Xt, thr)] for tag, m in models.items()}
    torch.cuda.synchronize()
    (mf, vf, kf), (ml, vl, kl) = res["fused"], res["layers"]
    for o in range(2):
        assert _rel(mf[:, o], ml[:, o]) <= 1e-3, o
        assert _rel(vf[:, o], vl[:, o]) <= 2e-2, o
    clear = np.abs(vl[:, 0] - thr) > 0.05 * thr
    assert np.array_equal(kf[clear], kl[clear]) and kf.sum() > 0
    # FP64 forward of every member (oracle/mlp.py) on the same BF16 weights and inputs
    mean, inv_std, ymean, ystd = models["fused"].norm()
    xs = np.zeros((n, 16))
    xs[:, :7] = omlp.bf16((X - mean[:7].astype(np.float32)) * inv_std[:7].astype(np.float32))
    outs = []
    for e in range(4):
        layers = [(omlp.bf16(W), b.astype(np.float64)) for W, b in models["fused"].layers(flats[e])]
        _, _, out = omlp.loss_and_grads(layers, xs, Y.astype(np.float64), ymean, ystd)
        outs.append(np.stack([out[:, 0] * ystd + ymean, out[:, 1]], axis=1))
    ref = np.mean(outs, axis=0)
    for o in range(2):
        assert _rel(mf[:, o], ref[:, o]) <= 1e-2, o
    for m in models.values():
        m.close()


def test_screen_keeps_slow_growing_cells(sg):
    """A dense, slow beam (n_b/n_p = 0.087, gamma = 10.4, L = 81.5) grows by
    ~e^180 at its back over 1000 steps but only ~e^11 near its front: the
    solver fallback answers queries at the front with the labels' values
    (finite, equal to the labels drawn by qs_sur_points), not zeros."""
    import torch
    qs, sur = sg
    p = synth.scaled(synth.BATCH_BASE, nkx=12, nky=12, species=[(-1.0, 1.0, 0.0870664478545601)],
                     gamma_b=10.410552660460878, n_xi=3261, dxi=0.025, length=81.525)
    Xq, Yq, _ = sur.generate([p], [1000], 4000, seed=2, noise_seed=1)
    front = Xq[:, 3] < 10.0
    assert int(front.sum()) > 100 and bool(torch.isfinite(Yq).all())
    Xtr, Ytr, _ = sur.generate([p], [500, 1000], 4096, seed=1)
    m = sur.SurModel(Xtr, Ytr, epochs=1, batch=2048, ensemble=2, seed=3)
    m.set_threshold(-1.0)                       # every query goes to the solver
    y, v, mask, ns = m.screen([p], Xq, noise_seed=1)
    torch.cuda.synchronize()
    assert ns == Xq.shape[0] and bool(torch.isfinite(y).all())
    d = (y[:, 0] - Yq[:, 0]).abs()
    assert float(d.max()) <= 1e-3, float(d.max())
    assert float(Yq[front, 0].max()) < float(Yq[~front, 0].max()) - 50.0   # the dynamic range in play
    m.close()
