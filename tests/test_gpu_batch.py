"""GPU tests of the batching form through the C ABI: many uneven replicas stepped as one CUDA
graph launch per step reproduce, bitwise, each replica stepped on its own; the FP64 residual check
of the constant-potential conditions; the stream-width, Verlet-skin and structure-factor tile
autotuners restore state."""
import numpy as np
import pytest

from paper_2509_24742_gb300 import srbe, workloads as wl

pytestmark = pytest.mark.gpu
ALPHA_A = 1.7


def _replicas():
    """Three uneven MD slabs: different boxes, lattices, ion counts, voltages, P and M."""
    a = wl.make_slab("r0", (2.0, 2.0, 12.0), 8, 8, 60, 3, alpha=3.5, eta_inv=19.79, rc=1.2, P=50, M=2,
                     dpsi_volt=1.0, seed=21, ax=0.25, ay=0.25, with_md=True)
    b = wl.make_slab("r1", (2.5, 2.5, 10.0), 10, 10, 90, 3, alpha=3.5, eta_inv=19.79, rc=1.2, P=80, M=None,
                     dpsi_volt=2.5, seed=22, with_md=True, placement="lattice")
    c = wl.make_slab("r2", (2.0, 2.0, 16.0), 8, 8, 40, 1, alpha=3.5, eta_inv=19.79, rc=1.2, P=30, M=3,
                     dpsi_volt=0.0, seed=23, ax=0.25, ay=0.25, with_md=True)
    return [a, b, c]


SETUP = [(srbe.FP64, srbe.DIRECT), (srbe.MIXED, srbe.DIRECT), (srbe.MIXED, srbe.PCG)]
SEEDS = [101, 202, 303]


def _contexts(slabs):
    out = []
    for s, (prec, solver) in zip(slabs, SETUP):
        c = srbe.from_slab(s, precision=prec, alpha_A=ALPHA_A, md=True)
        if solver == srbe.PCG:
            c.set_solver(srbe.PCG, tol=1e-10, maxit=500, warm=srbe.WARM_PREVIOUS)
        out.append(c)
    return out


def _state(ctxs):
    return [c.get_positions(velocities=True) for c in ctxs]


def test_batch_is_bitwise_each_replica_alone():
    slabs = _replicas()
    solo = _contexts(slabs)
    for c, sd in zip(solo, SEEDS):
        c.step(2, sd)
        c.step(4, sd)
    ref = _state(solo)
    ref_q = [c.forces()[1] for c in solo]
    for c in solo:
        c.close()
    for width in (0, 2):
        ctxs = _contexts(slabs)
        with srbe.Batch(ctxs) as b:
            b.set_width(width)
            b.step(2, SEEDS)
            b.step(4, SEEDS)
            got = _state(ctxs)
        got_q = [c.forces()[1] for c in ctxs]
        for c in ctxs:
            c.close()
        for (r0, v0), (r1, v1) in zip(ref, got):
            assert np.array_equal(r0, r1) and np.array_equal(v0, v1)
        for q0, q1 in zip(ref_q, got_q):
            assert np.array_equal(q0, q1)


def test_residual_check_of_the_charges():
    slabs = _replicas()
    ctxs = _contexts(slabs)
    with srbe.Batch(ctxs) as b:
        res = b.step(3, SEEDS, residuals=True)
    single = [c.charge_residual() for c in ctxs]
    for c in ctxs:
        c.close()
    print("FP64 residuals of the charge solve: FP64 direct %.3g, mixed direct %.3g, mixed PCG %.3g" % tuple(res))
    assert np.array_equal(res, single)
    assert res[0] < 1e-12
    assert res[1] < 1e-8
    assert res[2] < 1e-9


def test_autotuners_restore_state_and_pick_a_candidate():
    slabs = _replicas()
    solo = _contexts(slabs)
    for c, sd in zip(solo, SEEDS):
        c.step(3, sd)
    ref = _state(solo)
    for c in solo:
        c.close()
    ctxs = _contexts(slabs)
    with srbe.Batch(ctxs) as b:
        t = b.autotune(2, SEEDS, widths=[0, 1, 3])
        assert set(t) == {0, 1, 3} and all(v > 0 for v in t.values())
        assert b.width() == min(t, key=t.get)
        sk = ctxs[0].autotune_skin(2, SEEDS[0], skins=(0.05, 0.1, 0.2))
        assert all(v > 0 for v in sk.values())
        assert ctxs[0].skin() == min(sk, key=sk.get)
        b.step(3, SEEDS)
        got = _state(ctxs)
    for c in ctxs:
        c.close()
    for s, (r0, v0), (r1, v1) in zip(slabs, ref, got):
        L = np.asarray(s.box[:2])
        d = r1 - r0
        d[:, :2] -= L * np.round(d[:, :2] / L)
        assert np.abs(d).max() < 1e-9
        assert np.abs(v1 - v0).max() < 1e-7


def test_tile_autotuners_restore_state_and_keep_the_fastest():
    """The structure-factor tile (blocks per SM its chunking keeps) picked by timing, for a batch and
    for one context: every candidate is timed, the fastest is kept, the MD state is restored, and the
    tile changes the forces only by summation order."""
    slabs = _replicas()
    ctxs = _contexts(slabs)
    with srbe.Batch(ctxs) as b:
        b.step(1, SEEDS)
        before = _state(ctxs)
        t = b.autotune_tiles(2, SEEDS, occ=(1, 4, 16))
        assert set(t) == {1, 4, 16} and all(v > 0 for v in t.values())
        assert all(c.tiles() == min(t, key=t.get) for c in ctxs)
        for (r0, v0), (r1, v1) in zip(before, _state(ctxs)):
            assert np.array_equal(r0, r1) and np.array_equal(v0, v1)
        one = ctxs[1].autotune_tiles(2, SEEDS[1], occ=(2, 8))
        assert set(one) == {2, 8} and ctxs[1].tiles() == min(one, key=one.get)
        res = b.step(2, SEEDS, residuals=True)
        assert np.all(res < 1e-8)
    # the FP64 replica's forces at the extreme tiles, same state and modes
    c = ctxs[0]
    F = {}
    for occ in (1, 16):
        c.set_tiles(occ)
        assert c.tiles() == occ
        c.sample_k(SEEDS[0], 7)
        F[occ] = c.forces()[0]
    assert np.linalg.norm(F[1] - F[16]) <= 1e-12 * np.linalg.norm(F[16])
    with pytest.raises(srbe.SrbeError):
        c.set_tiles(0)
    for c in ctxs:
        c.close()


def test_batch_errors():
    slabs = _replicas()[:2]
    c0 = srbe.from_slab(slabs[0], alpha_A=ALPHA_A, md=True)
    c1 = srbe.from_slab(slabs[1], alpha_A=ALPHA_A)          # no MD state
    with pytest.raises(srbe.SrbeError):
        srbe.Batch([c0, c0])
    with srbe.Batch([c0, c1]) as b:
        with pytest.raises(srbe.SrbeError) as e:
            b.step(1, [1, 2])
        assert e.value.code == srbe.SRBE_ESTATE
        with pytest.raises(ValueError):
            b.step(1, [1])
    c0.close()
    c1.close()


def test_batch_replicas_match_oracle(orc):
    """Each replica of a batch against the oracle's own trajectory (Algorithm 1, velocity Verlet,
    mode lists from the oracle's sampler with the replica's seed): the FP64 replica within 1e-9 nm,
    the mixed replicas (direct and PCG charge solve) within 1e-6 nm over the same 6 steps.  Every
    replica here starts from a random-sequential-addition packing (no two sites closer than d_min):
    a jittered-grid start without relaxation holds overlapping sites whose forces near 1e9
    kJ/mol/nm amplify FP32 rounding beyond any fixed bar within a few steps."""
    slabs = _replicas()
    slabs[1] = wl.make_slab("r1", (2.5, 2.5, 10.0), 10, 10, 60, 3, alpha=3.5, eta_inv=19.79, rc=1.2, P=80, M=None,
                            dpsi_volt=2.5, seed=22, with_md=True)
    ctxs = _contexts(slabs)
    with srbe.Batch(ctxs) as b:
        b.set_width(2)
        b.step(2, SEEDS)
        b.step(4, SEEDS)
        got = _state(ctxs)
    for c in ctxs:
        c.close()
    for s, seed, (prec, _), (r, v) in zip(slabs, SEEDS, SETUP, got):
        ref = orc.System(s, alpha_A=ALPHA_A)
        rr, vv = s.r.copy(), s.v.copy()
        m, c = ref.modes(orc.sample_metropolis(s.box, s.alpha, s.M, s.P, seed, 0))
        F = orc.evaluate(ref.at(rr), ref.factor, m, c)["F"]
        for step in range(1, 7):
            m, c = ref.modes(orc.sample_metropolis(s.box, s.alpha, s.M, s.P, seed, step))
            rr, vv, ev = ref.md_step(rr, vv, F, m, c)
            F = ev["F"]
        L = np.asarray(s.box[:2])
        d = r - rr
        d[:, :2] -= L * np.round(d[:, :2] / L)
        dv = np.linalg.norm(v - vv) / np.linalg.norm(vv)
        print("%s (%s): max |dr| %.2e nm, velocity rel err %.2e"
              % (s.name, "FP64" if prec == srbe.FP64 else "mixed", np.abs(d).max(), dv))
        if prec == srbe.FP64:
            assert np.abs(d).max() < 1e-9 and dv < 1e-8
        else:
            assert np.abs(d).max() < 1e-6 and dv < 1e-4
