"""Parity of the CUDA path (through the C ABI) with the CPU oracle on the same seeded inputs.

Bars: FP64 path within 1e-10 normwise relative on forces and charges (and psi_bar, b);
integer work (the mode sampler) bit-exact; the mixed form within RMS force error 1e-3 of the
FP64 GPU path.  Mode lists come from the oracle's sampler, never from the library."""
import numpy as np
import pytest

from paper_2509_24742_gb300 import srbe, workloads as wl

pytestmark = pytest.mark.gpu

ALPHA_A = 1.7          # A-build Ewald parameter shared by both sides (alpha_A (Lz - H) = 6.8)
TOL = 1e-10


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / (nb if nb > 0 else 1.0)


@pytest.fixture(scope="module")
def slab784():
    return wl.one_shot_784()


@pytest.fixture(scope="module")
def ref784(orc, slab784):
    return orc.System(slab784, alpha_A=ALPHA_A)


def gpu_ctx(slab, precision=srbe.FP64, alpha_A=ALPHA_A, md=False):
    return srbe.from_slab(slab, precision=precision, alpha_A=alpha_A, md=md)


def test_fp64_forces_charges_match_oracle(orc, slab784, ref784):
    samples = orc.sample_metropolis(slab784.box, slab784.alpha, slab784.M, slab784.P, 3001, 0)
    m, c = ref784.modes(samples)
    ev = ref784.evaluate(m, c, with_lj=False)
    with gpu_ctx(slab784) as ctx:
        ctx.set_k(samples)
        F, Q, psi, E = ctx.forces(energy=True)
        Q2, psi2, b = ctx.solve_charges()
    assert rel(F, ev["F"]) < TOL
    assert rel(Q, ev["Q"]) < TOL
    assert abs(psi * srbe.VOLT - ev["psi_bar"]) < TOL * abs(ev["psi_bar"])
    assert rel(b * srbe.VOLT, ev["b"]) < TOL
    assert np.array_equal(Q, Q2)
    assert abs(Q.sum()) < 1e-12 * np.abs(Q).sum()
    np.testing.assert_allclose(E[:6], ev["E"], rtol=1e-9, atol=1e-9 * np.abs(ev["E"]).max())


def test_full_ewald_mode_list_matches_oracle(orc, slab784, ref784):
    """The same kernels evaluate full Ewald (kmax 8 x 8 x 48) from an explicit mode list."""
    m = orc.full_modes(slab784.box, slab784.alpha, (8, 8, 48))
    c = orc.ewald_weight(slab784.box, slab784.alpha, m)
    ev = ref784.evaluate(m, c, with_lj=False)
    with gpu_ctx(slab784) as ctx:
        ctx.set_mode_list(m, c)
        F, Q, psi = ctx.forces()
    assert rel(F, ev["F"]) < TOL
    assert rel(Q, ev["Q"]) < TOL


def test_sampler_bit_exact_with_oracle(orc, slab784):
    with gpu_ctx(slab784) as ctx:
        for step in (0, 1, 17):
            ctx.sample_k(3001, step)
            m, G = ctx.get_k()
            ref = orc.sample_metropolis(slab784.box, slab784.alpha, slab784.M, slab784.P, 3001, step)
            assert np.array_equal(m, ref)
            assert abs(G - orc.G_closed(slab784.box, slab784.alpha, slab784.M)) < 1e-12 * G
        ctx.set_sampler(srbe.EXACT, (8, 8, 48))
        ctx.sample_k(5, 2)
        m, G = ctx.get_k()
        ref = orc.sample_exact(slab784.box, slab784.alpha, slab784.M, slab784.P, 5, 2, (8, 8, 48))
        assert np.array_equal(m, ref)
        assert abs(G - orc.G_closed(slab784.box, slab784.alpha, slab784.M, (8, 8, 48))) < 1e-12 * G


def test_mixed_precision_error_bounds(orc, slab784):
    samples = orc.sample_metropolis(slab784.box, slab784.alpha, slab784.M, slab784.P, 3001, 4)
    with gpu_ctx(slab784) as c64:
        c64.set_k(samples)
        F64, Q64, _ = c64.forces()
    with gpu_ctx(slab784, precision=srbe.MIXED) as c32:
        c32.set_k(samples)
        F32, Q32, _ = c32.forces()
    rms_f = np.sqrt(((F32 - F64) ** 2).sum(1).mean()) / np.sqrt((F64 ** 2).sum(1).mean())
    assert rms_f < 1e-3, rms_f
    assert rel(Q32, Q64) < 1e-3


@pytest.mark.parametrize("case", ["no_ions", "no_samples", "no_deterministic", "ragged"])
def test_edge_cases_match_oracle(orc, case):
    s = wl.one_shot_784()
    if case == "no_ions":
        s.r, s.q = np.zeros((0, 3)), np.zeros(0)
        s.mol, s.itype, s.mass = s.mol[:0], s.itype[:0], s.mass[:0]
    elif case == "ragged":
        keep = 2 * 67 + 1          # odd count, not a multiple of the 128-thread tiles
        s.r, s.q = s.r[:keep].copy(), s.q[:keep].copy()
        s.q -= s.q.mean()
        s.mol, s.itype, s.mass = s.mol[:keep], s.itype[:keep], s.mass[:keep]
    P = 0 if case == "no_samples" else 37
    M = 0 if case == "no_deterministic" else s.M
    s.P, s.M = P, M
    ref = orc.System(s, alpha_A=ALPHA_A)
    samples = orc.sample_metropolis(s.box, s.alpha, M, P, 11, 0) if P else np.zeros((0, 3), np.int32)
    m, c = ref.modes(samples)
    ev = ref.evaluate(m, c, with_lj=False)
    with gpu_ctx(s) as ctx:
        ctx.set_k(samples)
        F, Q, psi = ctx.forces()
    assert rel(Q, ev["Q"]) < TOL
    if s.n_ion:
        assert rel(F, ev["F"]) < TOL


def test_results_are_bitwise_reproducible(orc, slab784):
    samples = orc.sample_metropolis(slab784.box, slab784.alpha, slab784.M, slab784.P, 1, 1)
    out = []
    for _ in range(2):
        with gpu_ctx(slab784) as ctx:
            ctx.set_k(samples)
            out.append(ctx.forces())
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


def test_errors_are_reported(slab784):
    with srbe.Context(slab784.box, slab784.alpha, slab784.eta, slab784.rc, 10, 2) as ctx:
        with pytest.raises(srbe.SrbeError) as e:
            ctx.forces()
        assert e.value.code == srbe.SRBE_ESTATE
        ctx.set_electrode(slab784.R, slab784.side)
        with pytest.raises(srbe.SrbeError) as e:
            ctx.set_k(np.array([[0, 0, 1]]))      # inside I
        assert e.value.code == srbe.SRBE_EINVAL


@pytest.mark.parametrize("thermostat", [None, (5.0, 400.0, 17)])
def test_md_steps_match_oracle(orc, thermostat):
    """Algorithm 1 with velocity Verlet (and optionally the Langevin thermostat of Eq. 39): a few
    steps of the MD slab (3-site cations, LJ, bonds) on a reduced copy, with the mode list of each
    step drawn by the oracle's own sampler and the thermostat noise by the oracle's own generator."""
    s = wl.make_slab("md_small", (2.0, 2.0, 12.0), 8, 8, 60, 3, alpha=3.5, eta_inv=19.79, rc=1.2, P=50, M=2,
                     dpsi_volt=1.0, seed=21, ax=0.25, ay=0.25, with_md=True)
    seed, nsteps = 77, 4
    ref = orc.System(s, alpha_A=ALPHA_A)
    r, v = s.r.copy(), s.v.copy()
    m, c = ref.modes(orc.sample_metropolis(s.box, s.alpha, s.M, s.P, seed, 0))
    F = orc.evaluate(ref.at(r), ref.factor, m, c)["F"]
    for step in range(1, nsteps + 1):
        m, c = ref.modes(orc.sample_metropolis(s.box, s.alpha, s.M, s.P, seed, step))
        r, v, ev = ref.md_step(r, v, F, m, c, thermostat=thermostat, step=step)
        F = ev["F"]
    with gpu_ctx(s, md=True) as ctx:
        if thermostat:
            ctx.set_thermostat(*thermostat)
        ctx.step(nsteps, seed)
        rg, vg = ctx.get_positions(velocities=True)
    d = rg - r
    d[:, :2] -= np.asarray(s.box[:2]) * np.round(d[:, :2] / np.asarray(s.box[:2]))
    assert np.abs(d).max() < 1e-9
    assert rel(vg, v) < 1e-8


@pytest.mark.parametrize("precision,solver,thermo,lattice", [(srbe.FP64, srbe.DIRECT, 0.0, 0),
                                                             (srbe.MIXED, srbe.DIRECT, 5.0, 0),
                                                             (srbe.MIXED, srbe.PCG, 0.0, 0),
                                                             (srbe.FP64, srbe.DIRECT, 5.0, 2),
                                                             (srbe.MIXED, srbe.LATTICE, 5.0, 2)])
def test_graph_replay_is_bitwise_the_ordinary_path(precision, solver, thermo, lattice):
    """srbe_step replaying its captured CUDA graphs gives bitwise the trajectory of the ordinary
    launch path, across several calls, a read-back in between and a state change that recaptures."""
    s = wl.make_slab("md_small", (2.0, 2.0, 12.0), 8, 8, 60, 3, alpha=3.5, eta_inv=19.79, rc=1.2, P=50, M=2,
                     dpsi_volt=1.0, seed=21, ax=0.25, ay=0.25, with_md=True)
    out = []
    for graphs in (False, True):
        with srbe.from_slab(s, precision=precision, alpha_A=ALPHA_A, md=True) as ctx:
            ctx.set_graphs(graphs)
            ctx.set_thermostat(thermo, 400.0, 5)
            ctx.set_lattice(lattice)
            if solver == srbe.PCG:
                ctx.set_solver(srbe.PCG, tol=1e-10, maxit=500, warm=srbe.WARM_PREVIOUS)
            elif solver == srbe.LATTICE:
                ctx.set_solver(srbe.LATTICE)
            ctx.step(3, 91)
            r1, v1 = ctx.get_positions(velocities=True)
            ctx.step(5, 91)
            state = ctx.graph_state()
            ctx.set_solver(solver, tol=1e-10, maxit=500, warm=srbe.WARM_ZERO)   # drops the graphs
            ctx.step(4, 91)
            r2, v2 = ctx.get_positions(velocities=True)
            F, Q, psi = ctx.forces()
        out.append((r1, v1, r2, v2, F, Q, state))
    assert out[0][6] == (0, 0)
    assert out[1][6][0] == 1 and out[1][6][1] > 5
    for a, b in zip(out[0][:6], out[1][:6]):
        assert np.array_equal(a, b)


def test_split_force_pass_matches_single_pass():
    """The mixed form without energies runs the ion-ion pairs and bonds as their own pass on the side
    stream; with energies it runs one pass.  Same charges, same forces up to FP32 summation order."""
    s = wl.md_11072()
    with srbe.from_slab(s, precision=srbe.MIXED, md=True) as c:
        c.sample_k(5, 1)
        F_split, Q1, psi1 = c.forces()
        F_one, Q2, psi2, _ = c.forces(energy=True)
    assert np.array_equal(Q1, Q2) and psi1 == psi2
    assert rel(F_split, F_one) < 1e-6, rel(F_split, F_one)


@pytest.mark.parametrize("move", ["within_skin", "beyond_skin"])
def test_set_positions_reuses_lists_only_while_valid(orc, slab784, move):
    """srbe_set_positions with the same ions and charges keeps the Verlet lists; the per-step
    half-skin test rebuilds them when needed.  Either way the forces equal a fresh context's."""
    import copy
    samples = orc.sample_metropolis(slab784.box, slab784.alpha, slab784.M, slab784.P, 3001, 2)
    rng = np.random.default_rng(17)
    r_new = slab784.r.copy()
    if move == "within_skin":
        r_new += rng.uniform(-0.004, 0.004, size=r_new.shape)
    else:
        r_new[:60, :2] += rng.uniform(-0.6, 0.6, size=(60, 2))
    with gpu_ctx(slab784) as c:
        c.set_k(samples)
        c.forces()
        c.set_positions(r_new, slab784.q)
        F1, Q1, _ = c.forces()
    s2 = copy.copy(slab784)
    s2.r = r_new
    with gpu_ctx(s2) as c2:
        c2.set_k(samples)
        F2, Q2, _ = c2.forces()
    assert rel(F1, F2) < 1e-12 and rel(Q1, Q2) < 1e-12
