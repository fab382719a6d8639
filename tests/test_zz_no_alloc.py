"""srbe_structure_factor_noalloc: the allocation-free structure-factor entry point, for callers that
cannot allocate device memory (an engine that owns all GPU memory through its own pool, or code
that must not allocate while its pipeline runs).  The caller owns every buffer (here torch
allocates them, as such a caller's pool would); the library adds no allocation.

Its output is checked, through the C ABI, against what the existing context path reports for the
same configuration and mode list:
  * U_F = 1/2 sum_k c_k |S1 + S2|^2 against srbe_forces' energy term;
  * the far part of b rebuilt from S1 against srbe_solve_electrode_charges' b (with rc below every
    ion-electrode distance, so that b = b_F + b_slab exactly);
over two calls in a row (ions, then electrode sites) and a repeat of the first call; both outputs
also against the CPU oracle's structure factor.  Further cases: the largest mode list (8,192 modes)
over 1e5 particles, where the scratch array caps the chunk count and every chunk spans many
128-particle batches, against the oracle on a subset of modes; and a first call made on a
non-blocking stream in a fresh process (the one-time set-up must be complete before that stream's
kernels read the table).
This file is collected last so that a failure here comes after every other test has run."""
import copy
import math
import os
import subprocess
import sys

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
    from oracle import oracle as orc
    for S, pos, w in ((S1, slab.r, slab.q), (S2, slab.R, Q)):
        ref = orc.sfac(np.asarray(pos, float), np.asarray(w, float), m, L) @ [1, 1j]
        assert np.linalg.norm(S - ref) < TOL * np.linalg.norm(ref)

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


def test_noalloc_largest_mode_list_many_batches_per_chunk(orc):
    """K = 8192 modes over 100,003 particles: the 2 MiB scratch array holds 16 chunks of ~6,300
    particles each (a ragged last chunk and a ragged last batch)."""
    import torch
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(8192)
    L = np.array([3.0, 2.5, 11.0])
    n, K = 100_003, 8192
    r = rng.uniform(0, 1, size=(n, 3)) * L
    w = rng.choice([-0.78, 0.78], size=n)
    m = rng.integers(-12, 13, size=(K, 3)).astype(np.int32)
    m[np.all(m == 0, axis=1)] = (0, 0, 1)
    S_d = torch.empty((K, 2), dtype=torch.float64, device=dev)
    r_d = torch.tensor(r, device=dev)
    w_d = torch.tensor(w, device=dev)
    m_d = torch.tensor(m, device=dev)
    for _ in range(2):                     # two calls in a row: the second reuses the array
        S_d.fill_(float("nan"))
        srbe.structure_factor_noalloc(L, n, r_d.data_ptr(), w_d.data_ptr(), K, m_d.data_ptr(), S_d.data_ptr(),
                                      torch.cuda.current_stream(dev).cuda_stream)
        torch.cuda.synchronize()
        S = S_d.cpu().numpy()
        sub = np.concatenate([np.arange(64), rng.choice(K, 64, replace=False), [K - 1]])
        ref = orc.sfac(r, w, m[sub], L)
        assert np.linalg.norm(S[sub] - ref) < TOL * np.linalg.norm(ref)


_FIRST_CALL_ON_SIDE_STREAM = r"""
import sys, numpy as np, torch
sys.path.insert(0, %(root)r)
from paper_2509_24742_gb300 import srbe
dev = torch.device("cuda", 0)
rng = np.random.default_rng(3)
L = np.array([2.0, 2.0, 12.0]); n, K = 4000, 300
r = rng.uniform(0, 1, size=(n, 3)) * L; w = rng.normal(size=n)
m = rng.integers(-6, 7, size=(K, 3)).astype(np.int32); m[np.all(m == 0, axis=1)] = (1, 0, 0)
side = torch.cuda.Stream(dev)          # a pool stream: created non-blocking
with torch.cuda.stream(side):
    r_d = torch.tensor(r, device=dev); w_d = torch.tensor(w, device=dev); m_d = torch.tensor(m, device=dev)
    S_d = torch.empty((K, 2), dtype=torch.float64, device=dev)
side.synchronize()
srbe.structure_factor_noalloc(L, n, r_d.data_ptr(), w_d.data_ptr(), K, m_d.data_ptr(), S_d.data_ptr(),
                              side.cuda_stream)
side.synchronize()
kr = 2 * np.pi * r / L
ph = kr @ m.T.astype(float)
ref = np.stack([(w[:, None] * np.cos(ph)).sum(0), (w[:, None] * np.sin(ph)).sum(0)], 1)
err = np.linalg.norm(S_d.cpu().numpy() - ref) / np.linalg.norm(ref)
print("first call on a non-blocking stream: rel err %%.2e" %% err)
sys.exit(0 if err < 1e-10 else 1)
"""


def test_noalloc_first_call_on_a_nonblocking_stream():
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, "-c", _FIRST_CALL_ON_SIDE_STREAM % {"root": root}],
                         capture_output=True, text=True, timeout=600)
    print(out.stdout, out.stderr[-2000:])
    assert out.returncode == 0
