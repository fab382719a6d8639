"""Pins of the learned-form oracle: backpropagated gradients equal central finite differences of
the loss; descriptors of a single ion reduce to the closed-form Gaussian of its distance; the low-k_z
features equal exp(-i k Z) S(k) written out for two charges."""
import math

import numpy as np

from oracle import mlp


def random_params(seed=0):
    rng = np.random.default_rng(seed)
    p = mlp.unpack(np.zeros(sum(int(np.prod(s)) for _, s in mlp.SIZES)))
    flat = []
    for name, shape in mlp.SIZES:
        if name in ("xs", "ys"):
            flat.append(rng.uniform(0.5, 2.0, size=shape).ravel())
        else:
            flat.append(rng.normal(scale=0.2, size=shape).ravel())
    return np.concatenate(flat)


def test_backprop_matches_finite_differences():
    P = random_params(1)
    rng = np.random.default_rng(2)
    D = rng.normal(size=(7, mlp.N_IN))
    T = rng.normal(size=7)
    loss, g = mlp.loss_and_grad(P, D, T)
    h = 1e-6
    for idx in rng.choice(mlp.N_TRAIN, size=40, replace=False):
        Pp, Pm = P.copy(), P.copy()
        Pp[idx] += h
        Pm[idx] -= h
        fd = (mlp.loss_and_grad(Pp, D, T)[0] - mlp.loss_and_grad(Pm, D, T)[0]) / (2 * h)
        assert abs(fd - g[idx]) < 1e-6 * max(1.0, abs(g[idx])), (idx, fd, g[idx])
    # forward is consistent with the loss: o = (y - ym) / ys
    p = mlp.unpack(P)
    y = mlp.forward(P, D)
    t = (T - p["ym"][0]) / p["ys"][0]
    assert abs(np.mean(((y - p["ym"][0]) / p["ys"][0] - t) ** 2) - loss) < 1e-12


def test_descriptors_single_ion_closed_form():
    box = (3.0, 3.0, 10.0)
    R = np.array([[1.0, 1.0, 1.0]])
    r = np.array([[1.3, 1.4, 1.5]])
    q = np.array([0.5])
    D = mlp.descriptors(box, R, r, q, rc=1.2)
    dist = math.sqrt(0.3 ** 2 + 0.4 ** 2 + 0.5 ** 2)
    mu = 0.25 + np.arange(32) / 31.0
    np.testing.assert_allclose(D[0, :32], 0.5 * np.exp(-(dist - mu) ** 2 / (2 * 0.035 ** 2)), rtol=1e-13)
    assert np.all(D[0, 32:64] == 0)


def test_low_kz_features_written_out():
    box = (2.0, 2.0, 9.0)
    R = np.array([[0.1, 0.2, 0.3], [0.5, 0.5, 6.0]])
    r = np.array([[1.0, 1.0, 2.0], [1.5, 0.3, 4.0]])
    q = np.array([0.7, -0.7])
    D = mlp.descriptors(box, R, r, q, rc=0.5)
    for m in (1, 4, 8):
        kz = 2 * math.pi * m / 9.0
        for j in range(2):
            v = (q[0] * np.exp(1j * kz * (2.0 - R[j, 2])) + q[1] * np.exp(1j * kz * (4.0 - R[j, 2])))
            assert abs(D[j, 64 + 2 * (m - 1)] - v.real) < 1e-13
            assert abs(D[j, 65 + 2 * (m - 1)] - v.imag) < 1e-13
