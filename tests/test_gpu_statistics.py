"""Statistics of the GPU path over sampling seeds (Theorems 3.1-3.2, Remark 3.1).

Over a lattice box shared by the sampler (exact i.i.d. draws, G over the same box) and the Ewald
reference, the SRBE right-hand side is an unbiased estimator of the Ewald one, and the electrode
charges are linear in it, so their mean over seeds is the Ewald charges; their variance falls as
1/P; the deterministic low-|k_z| set I lowers the variance of the right-hand side b (Remark 3.1:
those modes carry most of the sampled weight in an elongated cell).  The reference charges come from the same GPU
path with the full deterministic mode list (itself checked against the oracle in
test_gpu_parity.py).  Seeds are fixed, so the outcome is deterministic."""
import copy
import math

import numpy as np
import pytest

from paper_2509_24742_gb300 import srbe, workloads as wl

pytestmark = pytest.mark.gpu
ALPHA_A = 1.7
MMAX = (8, 8, 48)


def _charges(slab, P, M, n, seed, rhs=False):
    """n draws of the electrode charges (or of b) with P sampled modes and |m_z| <= M deterministic."""
    s = copy.copy(slab)
    s.P, s.M = P, M
    out = []
    with srbe.from_slab(s, alpha_A=ALPHA_A) as c:
        c.set_sampler(srbe.EXACT, MMAX)
        for step in range(n):
            c.sample_k(seed, step)
            Q, _, b = c.solve_charges()
            out.append(b if rhs else Q)
    return np.array(out)


def test_gpu_charges_unbiased_and_variance_one_over_P(orc):
    s = wl.one_shot_784()
    m_full = orc.full_modes(s.box, s.alpha, MMAX)
    c_full = orc.ewald_weight(s.box, s.alpha, m_full)
    with srbe.from_slab(s, alpha_A=ALPHA_A) as c:
        c.set_mode_list(m_full, c_full)
        Q_ref, _, _ = c.solve_charges()
    n = 1000
    var = {}
    for P in (25, 100):
        Qs = _charges(s, P, s.M, n, 500 + P)
        z = (Qs.mean(0) - Q_ref) / (Qs.std(0, ddof=1) / math.sqrt(n))
        assert np.abs(z).max() < 4.5, np.abs(z).max()
        var[P] = Qs.var(0).mean()
    # quadrupling P divides the charge variance by 4 (sampling error of the ratio ~10 %)
    assert 3.2 < var[25] / var[100] < 4.8, var


def test_gpu_deterministic_modes_reduce_rhs_variance():
    s = wl.one_shot_784()
    v = {M: _charges(s, 50, M, 300, 77, rhs=True).var(0).mean() for M in (0, 6)}
    assert v[6] < 0.5 * v[0], v
