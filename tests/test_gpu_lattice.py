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
