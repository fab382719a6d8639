"""The mixed form's charge update (Eqs. 9-11 through the projected inverse held as (hi, lo) FP32
pairs, double-float products) against the oracle's Cholesky solve of the same right-hand side.

The library returns b alongside Q and psi_bar, so the oracle solves exactly the system the GPU
solved: what is left is the error of the double-float product (about 2^-48 per term) and of the
FP64 inverse, far inside the FP64 path's 1e-10 bar.  Electrode sizes: 54, 378, 858 and 1,152
sites (even counts take the kernel's 16-byte path), and 377 (one site removed: the odd-count
path)."""
import numpy as np
import pytest

from paper_2509_24742_gb300 import srbe, workloads as wl

pytestmark = pytest.mark.gpu
ALPHA_A = 1.7
TOL = 1e-10


def rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / (nb if nb > 0 else 1.0)


@pytest.mark.parametrize("nx,ny,drop", [(3, 3, 0), (7, 9, 0), (7, 9, 1), (13, 11, 0), (16, 12, 0)])
def test_mixed_update_matches_oracle_solve(orc, nx, ny, drop):
    s = wl.make_slab("mixed_solve", (2.4, 2.2, 12.0), nx, ny, 40, 1, alpha=3.5, eta_inv=19.79, rc=1.0, P=60, M=2,
                     dpsi_volt=1.5, seed=40 + nx)
    if drop:
        s.R, s.side = s.R[:-drop].copy(), s.side[:-drop].copy()
    assert s.n_ele == 6 * nx * ny - drop
    ref = orc.System(s, alpha_A=ALPHA_A)
    samples = orc.sample_metropolis(s.box, s.alpha, s.M, s.P, 77, 3)
    with srbe.from_slab(s, precision=srbe.MIXED, alpha_A=ALPHA_A) as ctx:
        ctx.set_k(samples)
        Q, psi, b = ctx.solve_charges()
        Q2, psi2, b2 = ctx.solve_charges()
        res = ctx.charge_residual()
    Q_ref, psi_ref = orc.cp_solve(ref.factor, s.side, s.dpsi, b * srbe.VOLT)
    assert rel(Q, Q_ref) < TOL
    assert abs(psi * srbe.VOLT - psi_ref) < TOL * abs(psi_ref)
    assert abs(Q.sum()) < 1e-12 * np.abs(Q).sum()
    # fixed-order reductions make the update bitwise reproducible
    assert np.array_equal(Q, Q2) and psi == psi2 and np.array_equal(b, b2)
    assert res < 1e-10
