"""Parity of the lattice-electrode path (per-layer 2D transforms for S2 and the far part of b)
with the CPU oracle's plain per-site sums, and with the library's own plain path."""
import numpy as np
import pytest

from paper_2509_24742_gb300 import srbe, workloads as wl

pytestmark = pytest.mark.gpu
ALPHA_A = 1.7
TOL = 1e-10


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / (nb if nb > 0 else 1.0)


@pytest.fixture(scope="module")
def lat_slab():
    # 2 x 3 layers of 10 x 8 sites (odd layers shifted by half a step in x), commensurate with the box
    return wl.make_slab("lat", (2.5, 2.0, 12.0), 10, 8, 120, 1, alpha=3.5, eta_inv=19.79, rc=1.2, P=100, M=2,
                        dpsi_volt=1.5, seed=31)


def test_lattice_is_recognised(lat_slab):
    with srbe.from_slab(lat_slab, alpha_A=ALPHA_A) as ctx:
        assert ctx.lattice_info() == (6, 10, 8)
    with srbe.from_slab(wl.one_shot_784(), alpha_A=ALPHA_A) as ctx:   # 0.246 nm spacing: not commensurate
        assert ctx.lattice_info() == (0, 0, 0)


@pytest.mark.parametrize("kind", ["srbe", "full"])
def test_lattice_path_matches_oracle_and_plain_path(orc, lat_slab, kind):
    ref = orc.System(lat_slab, alpha_A=ALPHA_A)
    if kind == "srbe":
        samples = orc.sample_metropolis(lat_slab.box, lat_slab.alpha, lat_slab.M, lat_slab.P, 4001, 0)
        m, c = ref.modes(samples)
    else:   # every mode of a truncated Ewald sum: |m_x| up to 2.4 nx, so every alias class occurs
        m = orc.full_modes(lat_slab.box, lat_slab.alpha, (12, 10, 40))
        c = orc.ewald_weight(lat_slab.box, lat_slab.alpha, m)
    ev = ref.evaluate(m, c, with_lj=False)
    out = {}
    for lattice in (True, False):
        with srbe.from_slab(lat_slab, alpha_A=ALPHA_A) as ctx:
            ctx.set_lattice(2 if lattice else 0)
            if kind == "srbe":
                ctx.set_k(samples)
            else:
                ctx.set_mode_list(m, c)
            F, Q, psi, E = ctx.forces(energy=True)
            _, _, b = ctx.solve_charges()
            out[lattice] = (F, Q, psi, b, E)
    F, Q, psi, b, E = out[True]
    assert rel(F, ev["F"]) < TOL
    assert rel(Q, ev["Q"]) < TOL
    assert rel(b * srbe.VOLT, ev["b"]) < TOL
    assert abs(psi * srbe.VOLT - ev["psi_bar"]) < TOL * abs(ev["psi_bar"])
    np.testing.assert_allclose(E[:6], ev["E"], rtol=1e-9, atol=1e-9 * np.abs(ev["E"]).max())
    F0, Q0, psi0, b0, E0 = out[False]
    assert rel(F, F0) < 1e-12 and rel(Q, Q0) < 1e-12 and rel(b, b0) < 1e-12


def test_lattice_mixed_form_error(lat_slab):
    res = {}
    for prec in (srbe.FP64, srbe.MIXED):
        with srbe.from_slab(lat_slab, precision=prec, alpha_A=ALPHA_A) as ctx:
            ctx.set_lattice(2)
            ctx.sample_k(7, 0)
            res[prec] = ctx.forces()
    F64, Q64, _ = res[srbe.FP64]
    F32, Q32, _ = res[srbe.MIXED]
    assert np.sqrt(((F32 - F64) ** 2).sum(1).mean() / (F64 ** 2).sum(1).mean()) < 1e-4
    assert rel(Q32, Q64) < 1e-5


def test_spectral_solve_matches_dense_solve_and_oracle(orc, lat_slab):
    """The block-circulant (spectral) charge solve equals the dense projected inverse and the oracle."""
    samples = orc.sample_metropolis(lat_slab.box, lat_slab.alpha, lat_slab.M, lat_slab.P, 4002, 0)
    ref = orc.System(lat_slab, alpha_A=ALPHA_A)
    m, c = ref.modes(samples)
    ev = ref.evaluate(m, c, with_lj=False)
    out = {}
    for solver in (srbe.DIRECT, srbe.LATTICE):
        for prec in (srbe.FP64, srbe.MIXED):
            with srbe.from_slab(lat_slab, precision=prec, alpha_A=ALPHA_A) as ctx:
                ctx.set_solver(solver)
                ctx.set_k(samples)
                F, Q, psi = ctx.forces()
                out[solver, prec] = (F, Q, psi, ctx.charge_residual())
    F, Q, psi, res = out[srbe.LATTICE, srbe.FP64]
    F0, Q0, psi0, _ = out[srbe.DIRECT, srbe.FP64]
    assert rel(Q, Q0) < 1e-12 and rel(F, F0) < 1e-12 and abs(psi - psi0) < 1e-12 * abs(psi0)
    assert rel(Q, ev["Q"]) < TOL and rel(F, ev["F"]) < TOL
    assert res < 1e-12
    Fm, Qm, _, resm = out[srbe.LATTICE, srbe.MIXED]
    assert rel(Qm, Q0) < 1e-5 and resm < 1e-12


def test_spectral_only_electrode_beyond_the_dense_limit(orc):
    """18,432 lattice sites (2 x 3 layers of 64 x 48): no dense A exists; the charges satisfy the
    constant-potential conditions row by row against the oracle's A (rows formed one by one)."""
    s = wl.make_slab("lat18k", (8.0, 6.0, 24.0), 64, 48, 150, 1, alpha=3.5, eta_inv=19.79, rc=1.2, P=60, M=3,
                     dpsi_volt=2.0, seed=41)
    assert s.n_ele == 18432
    samples = orc.sample_metropolis(s.box, s.alpha, s.M, s.P, 4003, 0)
    m, c = orc.srbe_modes(s.box, s.alpha, s.M, samples, orc.G_closed(s.box, s.alpha, s.M))
    with srbe.from_slab(s) as ctx:
        assert ctx.lattice_info() == (6, 64, 48)
        with pytest.raises(srbe.SrbeError):
            ctx.set_solver(srbe.DIRECT)
        ctx.set_k(samples)
        F, Q, psi = ctx.forces()
        _, _, b = ctx.solve_charges()
        res = ctx.charge_residual()
        alpha_A = ctx.alpha_A()
    assert res < 1e-12
    assert abs(Q.sum()) < 1e-10 * np.abs(Q).sum()
    rng = np.random.default_rng(1)
    rows = np.sort(rng.choice(s.n_ele, 12, replace=False))
    bv = b * srbe.VOLT
    assert rel(bv[rows], orc.sampled_b(s, m, c, rows)) < TOL
    d = np.where(s.side == 1, 0.5, -0.5)
    AQ = orc.A_rows(s.box, s.eta, s.R, alpha_A, Q, rows)
    r = AQ - (s.dpsi * d[rows] + bv[rows]) - psi * srbe.VOLT
    assert np.abs(r).max() < 1e-10 * np.abs(s.dpsi * d + bv).max()
    ions = np.sort(rng.choice(s.n_ion, 12, replace=False))
    assert rel(F[ions], orc.sampled_forces(s, m, c, Q, ions)) < TOL
