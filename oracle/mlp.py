"""CPU oracle of the learned warm start (TEST INFRASTRUCTURE ONLY; the library never imports it).

Plain FP64 numpy restatement of the per-electrode-site descriptors and of the MLP
80 -> 128 -> 128 -> 1 (SiLU) with standardised inputs and target, its mean-squared-error loss and
the gradient of that loss by backpropagation, in the parameter layout of the C ABI:
W1[128][80], b1[128], W2[128][128], b2[128], W3[128], b3, input mean[80], input spread[80],
target mean, target spread.

Descriptors of electrode site j: 32 Gaussian radial densities (centres 0.25 + b/31 nm, width
0.035 nm) of the positive ion charge and 32 of the negative ion charge, over every ion image within
rc; then Re, Im of exp(-i k Z_j) S1(k) for k = 2 pi m / L_z, m = 1..8, the lowest k_z modes of the
structure factor of Eq. 15.
"""
from __future__ import annotations

import math

import numpy as np

N_IN, N_H = 80, 128
SIZES = [("W1", (N_H, N_IN)), ("b1", (N_H,)), ("W2", (N_H, N_H)), ("b2", (N_H,)), ("W3", (N_H,)), ("b3", (1,)),
         ("xm", (N_IN,)), ("xs", (N_IN,)), ("ym", (1,)), ("ys", (1,))]
N_TRAIN = sum(int(np.prod(s)) for n, s in SIZES[:6])


def unpack(P):
    P = np.asarray(P, dtype=np.float64)
    out, o = {}, 0
    for name, shape in SIZES:
        k = int(np.prod(shape))
        out[name] = P[o:o + k].reshape(shape)
        o += k
    assert o == P.size
    return out


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(P, D):
    p = unpack(P)
    x = (np.asarray(D, np.float64) - p["xm"]) / p["xs"]
    h1 = silu(x @ p["W1"].T + p["b1"])
    h2 = silu(h1 @ p["W2"].T + p["b2"])
    o = h2 @ p["W3"] + p["b3"][0]
    return o * p["ys"][0] + p["ym"][0]


def loss_and_grad(P, D, T):
    """Mean of (o - t)^2 with t the standardised target; gradient of the trainable entries."""
    p = unpack(P)
    x = (np.asarray(D, np.float64) - p["xm"]) / p["xs"]
    t = (np.asarray(T, np.float64) - p["ym"][0]) / p["ys"][0]
    n = x.shape[0]
    z1 = x @ p["W1"].T + p["b1"]
    h1 = silu(z1)
    z2 = h1 @ p["W2"].T + p["b2"]
    h2 = silu(z2)
    o = h2 @ p["W3"] + p["b3"][0]
    err = o - t
    loss = float(np.mean(err ** 2))
    dout = 2.0 * err / n
    g = {"W3": h2.T @ dout, "b3": np.array([dout.sum()])}
    dz2 = np.outer(dout, p["W3"]) * silu_grad(z2)
    g["W2"] = dz2.T @ h1
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ p["W2"]) * silu_grad(z1)
    g["W1"] = dz1.T @ x
    g["b1"] = dz1.sum(0)
    flat = np.concatenate([g[name].ravel() for name, _ in SIZES[:6]])
    return loss, flat


def descriptors(box, R, r, q, rc):
    L = np.asarray(box, float)
    R = np.asarray(R, float)
    r = np.asarray(r, float)
    q = np.asarray(q, float)
    mu = 0.25 + np.arange(32) / 31.0
    s = 0.035
    nx, ny = int(math.ceil(rc / L[0])) + 1, int(math.ceil(rc / L[1])) + 1
    out = np.zeros((R.shape[0], N_IN))
    for j in range(R.shape[0]):
        d = R[j] - r
        d[:, 0] -= L[0] * np.floor(d[:, 0] / L[0] + 0.5)
        d[:, 1] -= L[1] * np.floor(d[:, 1] / L[1] + 0.5)
        for a in range(-nx, nx + 1):
            for b in range(-ny, ny + 1):
                dd = d + np.array([a * L[0], b * L[1], 0.0])
                dist = np.sqrt((dd ** 2).sum(1))
                sel = dist < rc
                for dist_i, q_i in zip(dist[sel], q[sel]):
                    g = abs(q_i) * np.exp(-(dist_i - mu) ** 2 / (2 * s * s))
                    if q_i > 0:
                        out[j, :32] += g
                    elif q_i < 0:
                        out[j, 32:64] += g
    for m in range(1, 9):
        kz = 2 * math.pi * m / L[2]
        S = np.sum(q * np.exp(1j * kz * r[:, 2]))
        f = np.exp(-1j * kz * R[:, 2]) * S
        out[:, 64 + 2 * (m - 1)] = f.real
        out[:, 64 + 2 * (m - 1) + 1] = f.imag
    return out
