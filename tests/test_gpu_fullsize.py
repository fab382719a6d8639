"""Checks at the full size of the precision-form slab (8 x 8 x 32 nm, 12,288 electrode sites,
87,712 ion sites, P = 500) and of the 1.2 M-particle slab: the oracle cannot solve for the charges at
these sizes, so the tests compare sampled outputs it can compute one by one (b on sampled electrode
sites, electrostatic forces on sampled ions for the charges the GPU found) and check properties that
hold at any size (neutrality, the FP64 residual of the constant-potential conditions, the mixed form
against FP64).  At 100k the charges are also checked against the oracle's rows of A on sampled
sites."""
import numpy as np
import pytest

from paper_2509_24742_gb300 import srbe, workloads as wl

pytestmark = pytest.mark.gpu


def rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def big():
    return wl.precision_100k()


def test_precision_100k_sampled_parity_and_properties(orc, big):
    L = big.box
    samples = orc.sample_metropolis(L, big.alpha, big.M, big.P, 5003, 0)
    m, c = orc.srbe_modes(L, big.alpha, big.M, samples, orc.G_closed(L, big.alpha, big.M))
    with srbe.from_slab(big, precision=srbe.FP64) as ctx:
        assert ctx.lattice_info() == (6, 64, 32)
        ctx.set_k(samples)
        F, Q, psi = ctx.forces()
        _, _, b = ctx.solve_charges()
        res64 = ctx.charge_residual()
        alpha_A = ctx.alpha_A()
        ctx.set_lattice(0)                      # the plain per-site sums at the same size
        F0, Q0, _ = ctx.forces()
        ctx.set_lattice(1)
        ctx.set_precision(srbe.MIXED)
        F32, Q32, _ = ctx.forces()
        res32 = ctx.charge_residual()
    assert res64 < 1e-11 and res32 < 1e-9
    assert abs(Q.sum()) < 1e-10 * np.abs(Q).sum()
    assert rel(F, F0) < 1e-11 and rel(Q, Q0) < 1e-11
    rng = np.random.default_rng(0)
    sites = np.sort(rng.choice(big.n_ele, 48, replace=False))
    ions = np.sort(rng.choice(big.n_ion, 48, replace=False))
    assert rel(b[sites] * srbe.VOLT, orc.sampled_b(big, m, c, sites)) < 1e-10
    assert rel(F[ions], orc.sampled_forces(big, m, c, Q, ions)) < 1e-10
    # the charges meet the constant-potential conditions A Q = dpsi d + b + psi_bar e (Eqs. 9-10)
    # row by row, with the rows of A formed by the oracle one at a time (Eq. 18)
    rows = np.sort(rng.choice(big.n_ele, 12, replace=False))
    d = np.where(big.side == 1, 0.5, -0.5)
    bv = b * srbe.VOLT
    AQ = orc.A_rows(L, big.eta, big.R, alpha_A, Q, rows)
    r = AQ - (big.dpsi * d[rows] + bv[rows]) - psi * srbe.VOLT
    assert np.abs(r).max() < 1e-10 * np.abs(big.dpsi * d + bv).max()
    rms_f = np.sqrt(((F32 - F) ** 2).sum(1).mean() / (F ** 2).sum(1).mean())
    rms_q = np.sqrt(((Q32 - Q) ** 2).mean() / (Q ** 2).mean())
    print("100k slab: FP64 residual %.2e, mixed residual %.2e, mixed RMS force err %.2e, charge err %.2e"
          % (res64, res32, rms_f, rms_q))
    assert rms_f < 1e-3 and rms_q < 1e-4


def test_large_1m_sampled_parity_and_properties(orc):
    """The 1.2 M-particle slab (24 x 24 x 60 nm, 98,304 lattice electrode sites, 1.1 M ion sites,
    P = 1000): beyond the dense limit, so the charges come from the spectral solve.  b on sampled
    sites and the electrostatic forces on sampled ions (for the charges the GPU found) against the
    oracle, one output at a time; neutrality; the FP64 residual of the constant-potential conditions
    in both forms; the mixed form against FP64.  (A row of A at this size would cost the oracle
    ~2e11 operations, so the rows-of-A check of the 100k test is not repeated here.)"""
    big = wl.large_1m()
    L = big.box
    samples = orc.sample_metropolis(L, big.alpha, big.M, big.P, 5005, 0)
    m, c = orc.srbe_modes(L, big.alpha, big.M, samples, orc.G_closed(L, big.alpha, big.M))
    with srbe.from_slab(big, precision=srbe.FP64) as ctx:
        assert ctx.lattice_info() == (6, 128, 128)
        ctx.set_k(samples)
        F, Q, psi = ctx.forces()
        _, _, b = ctx.solve_charges()
        res64 = ctx.charge_residual()
        ctx.set_precision(srbe.MIXED)
        F32, Q32, _ = ctx.forces()
        res32 = ctx.charge_residual()
    assert res64 < 1e-11 and res32 < 1e-9
    assert abs(Q.sum()) < 1e-10 * np.abs(Q).sum()
    rng = np.random.default_rng(1)
    sites = np.sort(rng.choice(big.n_ele, 24, replace=False))
    ions = np.sort(rng.choice(big.n_ion, 24, replace=False))
    assert rel(b[sites] * srbe.VOLT, orc.sampled_b(big, m, c, sites)) < 1e-10
    assert rel(F[ions], orc.sampled_forces(big, m, c, Q, ions)) < 1e-10
    rms_f = np.sqrt(((F32 - F) ** 2).sum(1).mean() / (F ** 2).sum(1).mean())
    rms_q = np.sqrt(((Q32 - Q) ** 2).mean() / (Q ** 2).mean())
    print("1.2M slab: FP64 residual %.2e, mixed residual %.2e, mixed RMS force err %.2e, charge err %.2e"
          % (res64, res32, rms_f, rms_q))
    assert rms_f < 1e-3 and rms_q < 1e-4
