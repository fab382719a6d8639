"""Failure reporting through the C ABI: an iterative charge solve that stops at maxit, non-finite
forces or charges, and a bounded wait for the device.

No GPU fault is provoked.  The PCG case runs the real solver with maxit = 1.  The non-finite cases
use the library's test aid (srbe_debug_inject_nonfinite), which overwrites one computed entry with a
NaN before the check runs.  It is placed so that no kernel moves a particle with a NaN force: for
srbe_step the NaN enters after the drift, in the force pass of the last step, and only the closing
half kick sees it; the context is then closed.  The timeout case keeps the context's stream busy
with ordinary torch work."""
import ctypes

import numpy as np
import pytest

from paper_2509_24742_gb300 import srbe, workloads as wl

pytestmark = pytest.mark.gpu
ALPHA_A = 1.7


def _slab():
    return wl.make_slab("md_small", (2.0, 2.0, 12.0), 8, 8, 60, 3, alpha=3.5, eta_inv=19.79, rc=1.2, P=50, M=2,
                        dpsi_volt=1.0, seed=21, ax=0.25, ay=0.25, with_md=True)


def _raw_forces(ctx):
    """srbe_forces through the C ABI with caller arrays: (status, F, Q, psi_bar)."""
    F = np.empty((ctx.n_ion, 3))
    Q = np.empty(ctx.n_ele)
    psi = ctypes.c_double()
    dp = ctypes.POINTER(ctypes.c_double)
    code = ctx.lib.srbe_forces(ctx.h, F.ctypes.data_as(dp), Q.ctypes.data_as(dp), ctypes.byref(psi), None)
    return code, F, Q, psi.value


@pytest.mark.parametrize("precision", [srbe.FP64, srbe.MIXED])
def test_pcg_at_maxit_reports_enotconv_and_falls_back_to_the_direct_solve(orc, precision):
    s = _slab()
    samples = orc.sample_metropolis(s.box, s.alpha, s.M, s.P, 5, 0)
    with srbe.from_slab(s, precision=precision, alpha_A=ALPHA_A, md=True) as direct:
        direct.set_k(samples)
        F_d, Q_d, psi_d = direct.forces()
    with srbe.from_slab(s, precision=precision, alpha_A=ALPHA_A, md=True) as direct:
        direct.step(3, 11)
        r_d, v_d = direct.get_positions(velocities=True)
    with srbe.from_slab(s, precision=precision, alpha_A=ALPHA_A, md=True) as ctx:
        ctx.set_solver(srbe.PCG, tol=1e-12, maxit=1, warm=srbe.WARM_ZERO)
        ctx.set_k(samples)
        code, F, Q, psi = _raw_forces(ctx)
        assert code == srbe.SRBE_ENOTCONV
        assert b"maxit" in ctx.lib.srbe_last_error(ctx.h)
        assert ctx.solver_stats()[0] == 1
        # the outputs of that call are the direct solve's, bitwise
        assert np.array_equal(Q, Q_d) and psi == psi_d and np.array_equal(F, F_d)
        # the flag was reported once: the next call with a converging solve is clean
        ctx.set_solver(srbe.PCG, tol=1e-12, maxit=1000, warm=srbe.WARM_ZERO)
        ctx.forces()
        # MD: every step falls back, so the trajectory is the direct solve's, and the flag of the
        # asynchronous steps comes back from srbe_synchronize
        ctx.set_solver(srbe.PCG, tol=1e-12, maxit=1, warm=srbe.WARM_ZERO)
        ctx.set_positions(s.r, s.q)
        ctx.set_md(s.mass, s.itype, s.mol, *s.lj_tables(), s.bonds, s.bond_r0, s.bond_k, s.dt, v=s.v)
        ctx.step(3, 11)
        with pytest.raises(srbe.SrbeError) as e:
            ctx.synchronize()
        assert e.value.code == srbe.SRBE_ENOTCONV
        ctx.synchronize()                      # reported and cleared
        r, v = ctx.get_positions(velocities=True)
    assert np.array_equal(r, r_d) and np.array_equal(v, v_d)


@pytest.mark.parametrize("what", [1, 2])
def test_nonfinite_force_or_charge_is_reported(what):
    s = _slab()
    with srbe.from_slab(s, alpha_A=ALPHA_A, md=True) as ctx:
        ctx.sample_k(3, 0)
        ctx.forces()                           # clean
        ctx.debug_inject_nonfinite(what)
        code, F, Q, _ = _raw_forces(ctx)
        assert code == srbe.SRBE_ENONFINITE
        msg = ctx.lib.srbe_last_error(ctx.h)
        assert (b"forces" in msg) if what == 1 else (b"charges" in msg)
        # the outputs show what the check saw
        assert not np.isfinite(F).all()
        if what == 2:
            assert np.isnan(Q[0])
            with pytest.raises(srbe.SrbeError) as e:
                ctx.solve_charges()
            assert e.value.code == srbe.SRBE_ENONFINITE
        ctx.debug_inject_nonfinite(0)
        ctx.forces()                           # clean again


def test_nonfinite_force_in_an_md_step_is_reported():
    s = _slab()
    with srbe.from_slab(s, alpha_A=ALPHA_A, md=True) as ctx:
        ctx.step(2, 7)
        ctx.synchronize()                      # clean
        ctx.debug_inject_nonfinite(1)          # NaN in F[0] of the next step's force pass
        ctx.step(1, 7)
        with pytest.raises(srbe.SrbeError) as e:
            ctx.synchronize()
        assert e.value.code == srbe.SRBE_ENONFINITE
        _, v = ctx.get_positions(velocities=True)
        assert np.isnan(v[0]).any() and np.isfinite(v[1:]).all()


def test_batch_reports_a_replica_flag():
    slabs = [_slab(), wl.make_slab("r2", (2.0, 2.0, 16.0), 8, 8, 40, 1, alpha=3.5, eta_inv=19.79, rc=1.2, P=30, M=3,
                                   dpsi_volt=0.0, seed=23, ax=0.25, ay=0.25, with_md=True)]
    ctxs = [srbe.from_slab(sl, alpha_A=ALPHA_A, md=True) for sl in slabs]
    with srbe.Batch(ctxs) as b:
        b.step(1, [1, 2])
        ctxs[1].debug_inject_nonfinite(1)
        b.step(1, [1, 2])                      # the NaN enters after the drift; the closing kick flags it
        with pytest.raises(srbe.SrbeError) as e:
            b.step(1, [1, 2])
        assert e.value.code == srbe.SRBE_ENONFINITE
        assert "replica 1" in str(e.value)
    for c in ctxs:
        c.close()


def test_synchronize_times_out_while_the_stream_is_busy():
    import torch
    s = _slab()
    st = torch.cuda.Stream()
    with srbe.from_slab(s, alpha_A=ALPHA_A) as ctx:
        ctx.set_stream(st.cuda_stream)
        with torch.cuda.stream(st):
            x = torch.randn(4096, 4096, device="cuda")
            for _ in range(200):               # ~a second of queued work on the context's stream
                x = torch.tanh(x @ x * 1e-3)
        with pytest.raises(srbe.SrbeError) as e:
            ctx.synchronize(0.01)
        assert e.value.code == srbe.SRBE_ETIMEOUT
        ctx.synchronize(-1.0)
        assert st.query()
