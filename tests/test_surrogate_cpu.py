"""CPU pins of the surrogate references: FP64 backprop against central
finite differences, the GELU derivative, BF16 rounding, and the targets:
the class rule against the exact Green's function's CFI / OTSI regions
(front of the beam vs behind the transition xi_tr = C_cr Gamma tau)."""
import math

import numpy as np

import oracle
import synth
from oracle import mlp
from oracle import surdata


def _net(rng, sizes):
    return [(rng.standard_normal((o, i)) / np.sqrt(i), 0.1 * rng.standard_normal(o))
            for i, o in zip(sizes[:-1], sizes[1:])]


def test_backprop_matches_finite_differences():
    rng = np.random.default_rng(0)
    layers = _net(rng, [7, 12, 12, 2])
    X = rng.standard_normal((9, 7))
    Y = np.stack([rng.standard_normal(9), (rng.random(9) > 0.5).astype(float)], axis=1)
    _, grads, _ = mlp.loss_and_grads(layers, X, Y, ymean=0.3, ystd=1.7)
    eps = 1e-6
    for l, (W, b) in enumerate(layers):
        for arr, g in ((W, grads[l][0]), (b, grads[l][1])):
            flat = arr.reshape(-1)
            gf = g.reshape(-1)
            for idx in rng.choice(flat.size, min(12, flat.size), replace=False):
                old = flat[idx]
                flat[idx] = old + eps
                lp, _, _ = mlp.loss_and_grads(layers, X, Y, 0.3, 1.7)
                flat[idx] = old - eps
                lm, _, _ = mlp.loss_and_grads(layers, X, Y, 0.3, 1.7)
                flat[idx] = old
                fd = (lp - lm) / (2 * eps)
                assert abs(fd - gf[idx]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9


def test_gelu_derivative_and_bf16():
    z = np.linspace(-6, 6, 101)
    fd = (mlp.gelu(z + 1e-6) - mlp.gelu(z - 1e-6)) / 2e-6
    assert np.max(np.abs(fd - mlp.dgelu(z))) < 1e-8
    assert mlp.bf16(np.array([1.0, 1.00390625, 1.01171875]))[1] == 1.0        # tie -> even
    x = np.random.default_rng(1).standard_normal(1000)
    assert np.max(np.abs(mlp.bf16(x) - x) / np.abs(x)) <= 2.0 ** -8


def test_envelope_target_definition():
    dxi, A = 0.025, 1e-6
    mag = np.ones((5, 400))
    mag[0] = np.exp(0.3 * (np.arange(400) + 0.5) * dxi) * A
    y0, _ = surdata.targets(mag, dxi, 200, A)
    assert y0 == np.log(np.sqrt(np.mean(mag[0, 160:241] ** 2))) - np.log(A)


def test_class_rule_on_the_impulse_response():
    """Impulse response of Eq. (18): non-oscillatory (CFI, label 0) ahead of
    the transition xi_tr = C_cr Gamma tau (Sec. III.B), oscillatory (OTSI,
    label 1) well behind it.  The label flips within ~1-2.5 xi_tr, where
    both coexist (transition region), so only the two sides are asserted."""
    G, D = 0.1, 0.025
    n0 = 0.01
    gam = n0 / G ** 2                        # Gamma^2 = n0/gamma for k >> 1
    for steps in (240, 400):
        p = synth.scaled(synth.SLAB_2D, species=[(-1.0, 1.0, n0)], gamma_b=gam, model="reduced",
                         n_xi=1600, dxi=D, length=40.0, dt=0.5, k_list=[1e4])
        nb, th = oracle.seed_impulse(p)
        oracle.sweep(p, nb, th, 0, steps)
        f = oracle.fields(p, nb)["mag"][:, 0, :]
        xi_tr = 0.3849 * G * steps * 0.5
        xs = np.arange(0.5, 39.0, 0.75)
        lab = np.array([surdata.targets(f, D, int(x / D), 1.0)[1] for x in xs])
        assert np.all(lab[xs <= 0.75 * xi_tr] == 0.0), steps
        assert np.all(lab[(xs >= 2.5 * xi_tr) & (xs <= 36.0)] == 1.0), steps
        assert math.isfinite(xi_tr)
