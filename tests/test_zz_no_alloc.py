"""srbe_structure_factor_noalloc: the allocation-free structure-factor entry point, for callers that
cannot allocate device memory (an engine that owns all GPU memory through its own pool, or code
that must not allocate while its pipeline runs).  The caller owns every buffer (here torch
allocates them, as such a caller's pool would); the library adds no allocation.

Its output is checked, through the C ABI, against what the existing context path reports for the
same configuration and mode list:
  * U_F = 1/2 sum_k c_k |S1 + S2|^2 against srbe_forces' energy term;
  * the far part of b rebuilt from S1 against srbe_solve_electrode_charges' b (with rc below every
    ion-electrode distance, so that b = b_F + b_slab exactly);
over two calls in a row (ions, then electrode sites) and a repeat of the first call.
This file is collected last so that a failure here comes after every other test has run."""
import copy
import math

import numpy as np
import pytest

from paper_2509_24742_gb300 import srbe, workloads as wl

pytestmark = pytest.mark.gpu
TOL = 1e-10


def test_noalloc_structure_factor_matches_existing_entry_points():
    import torch
    dev = torch.device("cuda", 0)
    slab = copy.copy(wl.one_shot_784())
    slab.rc = 0.25                      # every ion-electrode distance is >= 0.3 nm: no near part in b
    L = np.asarray(slab.box)
    V = float(np.prod(L))
    with srbe.from_slab(slab, precision=srbe.FP64, alpha_A=1.7) as ctx:
        ctx.sample_k(4242, 3)
        samples, G = ctx.get_k()
        F, Q, psi, E = ctx.forces(energy=True)
        Qb, _, b_volt = ctx.solve_charges()
    assert np.array_equal(Q, Qb)

    # the context's mode list: I folded to +m_z with twice the Ewald weight, then the samples
    det = np.array([[0, 0, mz] for mz in range(1, slab.M + 1)], np.int32)
    m = np.concatenate([det, samples]).astype(np.int32)
    k2 = ((2 * math.pi * m / L) ** 2).sum(1)
    c = np.where(np.arange(m.shape[0]) < slab.M,
                 2 * 4 * math.pi / (V * k2) * np.exp(-k2 / (4 * slab.alpha ** 2)),
                 (G / slab.P) * 4 * math.pi / (V * k2))
    K = m.shape[0]

    r_d = torch.tensor(slab.r, dtype=torch.float64, device=dev)
    q_d = torch.tensor(slab.q, dtype=torch.float64, device=dev)
    R_d = torch.tensor(slab.R, dtype=torch.float64, device=dev)
    Q_d = torch.tensor(Q, dtype=torch.float64, device=dev)
    m_d = torch.tensor(m, dtype=torch.int32, device=dev)
    S1_d = torch.empty((K, 2), dtype=torch.float64, device=dev)
    S2_d = torch.empty((K, 2), dtype=torch.float64, device=dev)
    S1b_d = torch.empty((K, 2), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev).cuda_stream

    # two calls in a row, then the first again
    srbe.structure_factor_noalloc(L, slab.n_ion, r_d.data_ptr(), q_d.data_ptr(), K, m_d.data_ptr(),
                                  S1_d.data_ptr(), stream)
    srbe.structure_factor_noalloc(L, slab.n_ele, R_d.data_ptr(), Q_d.data_ptr(), K, m_d.data_ptr(),
                                  S2_d.data_ptr(), stream)
    srbe.structure_factor_noalloc(L, slab.n_ion, r_d.data_ptr(), q_d.data_ptr(), K, m_d.data_ptr(),
                                  S1b_d.data_ptr(), stream)
    torch.cuda.synchronize()
    S1 = S1_d.cpu().numpy() @ [1, 1j]
    S2 = S2_d.cpu().numpy() @ [1, 1j]
    assert np.array_equal(S1_d.cpu().numpy(), S1b_d.cpu().numpy())

    # U_F of the existing srbe_forces (kJ/mol) from the two outputs
    UF = 0.5 * float((c * np.abs(S1 + S2) ** 2).sum()) * srbe.K_E
    assert abs(UF - E[3]) < TOL * abs(E[3])

    # b of the existing srbe_solve_electrode_charges (V) from S1: b_F (Eq. 24) + slab term
    ph = (2 * math.pi * slab.R / L) @ m.T.astype(float)        # [n_ele, K]
    bF = -(c[None, :] * (np.cos(ph) * S1.real + np.sin(ph) * S1.imag)).sum(1)
    bS = -(4 * math.pi / V) * slab.R[:, 2] * float(slab.q @ slab.r[:, 2])
    b_ref = b_volt * srbe.VOLT
    assert np.linalg.norm(bF + bS - b_ref) < TOL * np.linalg.norm(b_ref)


def test_noalloc_rejects_oversized_mode_lists():
    import torch
    from paper_2509_24742_gb300 import srbe as S
    dev = torch.device("cuda", 0)
    m = torch.zeros((8193, 3), dtype=torch.int32, device=dev)
    out = torch.empty((8193, 2), dtype=torch.float64, device=dev)
    r = torch.zeros((1, 3), dtype=torch.float64, device=dev)
    with pytest.raises(S.SrbeError) as e:
        S.structure_factor_noalloc((1.0, 1.0, 1.0), 1, r.data_ptr(), r.data_ptr(), 8193, m.data_ptr(),
                                   out.data_ptr())
    assert e.value.code == S.SRBE_EINVAL
