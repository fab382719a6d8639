"""The captured host-I/O force provider (srbe_set_host_io / srbe_forces_host_io) against the
uncaptured host-pointer calls it stands for: srbe_set_positions with the same charges, then
srbe_sample_k(seed, step) and srbe_forces.  Both forms, several consecutive frames of an MD
trajectory (so that the Verlet lists age and get rebuilt), a state change that recaptures, and a
non-finite position in the input buffer."""
import numpy as np
import pytest

from paper_2509_24742_gb300 import srbe, workloads as wl

pytestmark = pytest.mark.gpu
ALPHA_A = 1.7


def _slab():
    return wl.make_slab("md_small", (2.0, 2.0, 12.0), 8, 8, 60, 3, alpha=3.5, eta_inv=19.79, rc=1.2, P=50, M=2,
                        dpsi_volt=1.0, seed=21, ax=0.25, ay=0.25, with_md=True)


def _frames(s, n):
    """n consecutive frames of the context's own MD trajectory (20 steps apart)."""
    out = []
    with srbe.from_slab(s, precision=srbe.FP64, alpha_A=ALPHA_A, md=True) as c:
        for _ in range(n):
            c.step(20, 5)
            out.append(c.get_positions())
    return out


@pytest.mark.parametrize("precision", [srbe.FP64, srbe.MIXED])
def test_provider_is_bitwise_the_host_pointer_calls(precision):
    import torch
    s = _slab()
    frames = _frames(s, 5)
    r_h = torch.empty((s.n_ion, 3), dtype=torch.float64).pin_memory()
    F_h = torch.empty((s.n_ion, 3), dtype=torch.float64).pin_memory()
    Q_h = torch.empty(s.n_ele, dtype=torch.float64).pin_memory()
    ref, got = [], []
    with srbe.from_slab(s, precision=precision, alpha_A=ALPHA_A, md=True) as c:
        for t, r in enumerate(frames):
            c.set_positions(r, s.q)
            c.sample_k(77, t)
            ref.append(c.forces())
    with srbe.from_slab(s, precision=precision, alpha_A=ALPHA_A, md=True) as c:
        c.set_host_io(r_h.data_ptr(), F_h.data_ptr(), Q_h.data_ptr())
        for t, r in enumerate(frames):
            if t == 3:
                c.set_thermostat(0.0, 0.0, 0)          # a state change between calls: recapture
            r_h.numpy()[:] = r
            psi = c.forces_host_io(77, t)
            got.append((F_h.numpy().copy(), Q_h.numpy().copy(), psi))
    for (F0, Q0, p0), (F1, Q1, p1) in zip(ref, got):
        assert np.array_equal(F0, F1) and np.array_equal(Q0, Q1) and p0 == p1


def test_provider_rejects_unpinned_buffers_and_reports_bad_input():
    import torch
    s = _slab()
    r_h = torch.empty((s.n_ion, 3), dtype=torch.float64).pin_memory()
    F_h = torch.empty((s.n_ion, 3), dtype=torch.float64).pin_memory()
    plain = np.empty((s.n_ion, 3))
    with srbe.from_slab(s, alpha_A=ALPHA_A, md=True) as c:
        with pytest.raises(srbe.SrbeError) as e:
            c.forces_host_io(1, 0)
        assert e.value.code == srbe.SRBE_ESTATE
        with pytest.raises(srbe.SrbeError) as e:
            c.set_host_io(plain.ctypes.data, F_h.data_ptr())
        assert e.value.code == srbe.SRBE_EINVAL
        c.set_host_io(r_h.data_ptr(), F_h.data_ptr())
        r_h.numpy()[:] = s.r
        c.forces_host_io(1, 0)
        r_h.numpy()[5, 1] = np.nan
        with pytest.raises(srbe.SrbeError) as e:
            c.forces_host_io(1, 1)
        assert e.value.code == srbe.SRBE_EINVAL
        r_h.numpy()[:] = s.r
        c.forces_host_io(1, 2)
        assert np.isfinite(F_h.numpy()).all()
