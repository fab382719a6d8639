"""Pins of the oracle's Langevin thermostat (Eq. 39 with gamma read as a collision rate): the
counter-based noise is standard normal and reproducible, the exact Ornstein-Uhlenbeck step keeps
the Maxwell distribution at T and decays velocities by e^{-gamma dt}, and gamma = 0 is plain
velocity Verlet."""
import math

import numpy as np
import pytest
from scipy import stats


def test_noise_is_standard_normal_and_counter_based(orc):
    g = orc.langevin_gauss(11, 5, 40000)
    assert g.shape == (40000, 3)
    for a in range(3):
        assert abs(g[:, a].mean()) < 0.02
        assert abs(g[:, a].var() - 1.0) < 0.03
        assert stats.kstest(g[:, a], "norm").pvalue > 1e-3
    c = np.corrcoef(g.T)
    assert np.abs(c - np.eye(3)).max() < 0.03
    # the same (seed, step, ion) gives the same numbers whatever n; other steps and seeds differ
    assert np.array_equal(orc.langevin_gauss(11, 5, 100), g[:100])
    assert np.abs(orc.langevin_gauss(11, 6, 100) - g[:100]).min() > 0
    assert not np.allclose(orc.langevin_gauss(12, 5, 100), g[:100])
    # Philox word layout: ion i of step n uses counter (n, i, 0, 0) and key (seed, 'LANG')
    w = orc.philox4x64([5, 7, 0, 0], [11, 0x4C414E47])
    u = ((w >> np.uint64(11)).astype(np.float64) + 0.5) * 2.0 ** -53
    r0 = math.sqrt(-2 * math.log(u[0]))
    assert g[7, 0] == pytest.approx(r0 * math.cos(2 * math.pi * u[1]), rel=1e-15)
    assert g[7, 1] == pytest.approx(r0 * math.sin(2 * math.pi * u[1]), rel=1e-15)


def test_ou_step_keeps_maxwell_and_decays_at_gamma(orc):
    n, T, gamma, dt = 4000, 400.0, 5.0, 0.02
    mass = np.where(np.arange(n) % 2 == 0, 15.0, 145.0)
    v = np.zeros((n, 3))
    for step in range(120):                       # 12 relaxation times
        v = orc.langevin_o(v, mass, gamma, T, dt, 3, step)
    Tk = (mass[:, None] * v ** 2).sum() / (3 * n * orc.KB)
    assert abs(Tk - T) < 0.05 * T
    # E[v' | v] = e^{-gamma dt} v: regression slope over many particles
    v2 = orc.langevin_o(v, mass, gamma, T, dt, 3, 999)
    slope = (v * v2).sum() / (v * v).sum()
    assert slope == pytest.approx(math.exp(-gamma * dt), abs=0.02)
    # the per-particle kinetic energy is mass independent (equipartition)
    ke = 0.5 * mass[:, None] * v2 ** 2
    assert abs(ke[0::2].mean() - ke[1::2].mean()) < 0.1 * ke.mean()
    # gamma = 0 leaves velocities untouched
    assert np.array_equal(orc.langevin_o(v, mass, 0.0, T, dt, 3, 1), v)


def test_md_step_with_zero_friction_is_velocity_verlet(orc):
    from paper_2509_24742_gb300 import workloads as wl
    s = wl.tiny_slab(n_pairs=4)
    s.mass = np.full(s.n_ion, 40.0)
    ref = orc.System(s, alpha_A=2.5)
    m, c = ref.modes(orc.sample_metropolis(s.box, s.alpha, s.M, s.P, 1, 1))
    F = orc.evaluate(ref.at(s.r), ref.factor, m, c, with_lj=False)["F"]
    v0 = np.zeros((s.n_ion, 3))
    a = ref.md_step(s.r.copy(), v0, F, m, c)
    b = ref.md_step(s.r.copy(), v0, F, m, c, thermostat=(0.0, 300.0, 9), step=1)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    t = ref.md_step(s.r.copy(), v0, F, m, c, thermostat=(2.0, 300.0, 9), step=1)
    assert np.array_equal(t[0], a[0]) and not np.array_equal(t[1], a[1])
