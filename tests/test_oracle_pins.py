"""Pins of the CPU oracle against facts fixed by the paper and by mathematics,
independent of the oracle's own formulas:

* finite differences of the total energy (Eqs. 13, 16, 17) give Psi = A Q - b
  (Eq. 6) and the Hessian A (Eq. 18): pins every term of A and b, including the
  slab-term readings (4 pi / V) Z_i Z_j and -(4 pi Z_j / V) sum q_i z_i;
* finite differences of the energy give the forces (Eqs. 13, 21, slab term);
* the Ewald split is exact: energy, forces and A do not depend on alpha;
* the Ewald3D + slab-correction energy (Eq. 16 + Eq. 17) converges, as the
  vacuum padding grows, to the exact quasi-2D energy of Eq. 14, whose k_z
  integral is done here by adaptive quadrature;
* the self term of A is the R -> 0 limit of the electrode-electrode kernel;
* the constant-potential solution is neutral, has Psi = psi_bar -/+ dpsi / 2
  (Eqs. 7-11), and is antisymmetric for a mirror-antisymmetric cell.
"""
import copy
import math

import numpy as np
import pytest
import scipy.integrate

from paper_2509_24742_gb300 import workloads as wl


def converged_tiny(orc, alpha=2.0, **kw):
    s = wl.tiny_slab(alpha=alpha, **kw)
    s.rc = orc.A_rcut(alpha, 1e-17)
    return s


def total_energy(orc, s, Q, modes=None):
    """U_c = U_N + U_F - U_corr (Eqs. 13, 16, 17) in Gaussian units, full Ewald, fixed Q."""
    m = orc.A_modes(s.box, s.alpha, 1e-17) if modes is None else modes
    c = orc.ewald_weight(s.box, s.alpha, m)
    ev = orc.evaluate(s, None, m, c, Q_fixed=Q, with_lj=False)
    return ev["E"].sum() / orc.K_E, ev


def full_b(orc, s, m):
    c = orc.ewald_weight(s.box, s.alpha, m)
    S1 = orc.sfac(s.r, s.q, m, s.box)
    return orc.b_far(s.R, m, c, S1, s.box) + orc.b_near(s.box, s.alpha, s.eta, s.rc, s.r, s.q, s.R) \
        + orc.b_slab(s.box, s.r, s.q, s.R)


def test_potential_is_gradient_of_energy(orc):
    """Psi_j = dU/dQ_j = (A Q - b)_j (Eq. 6) with A from Eq. 18, for non-neutral perturbations
    too (A and the energy at the same alpha, see test_A_alpha_dependence_is_background_only)."""
    s = converged_tiny(orc)
    rng = np.random.default_rng(5)
    Q = rng.normal(scale=0.1, size=s.n_ele)
    Q -= Q.mean()
    m = orc.A_modes(s.box, s.alpha, 1e-17)
    A = orc.build_A(s.box, s.eta, s.R, alpha_A=s.alpha)
    b = full_b(orc, s, m)
    psi = A @ Q - b
    h = 1e-3
    for j in [0, 5, 11, 12, 23]:
        e = np.zeros(s.n_ele)
        e[j] = h
        up, _ = total_energy(orc, s, Q + e, m)
        dn, _ = total_energy(orc, s, Q - e, m)
        fd = (up - dn) / (2 * h)
        assert abs(fd - psi[j]) < 1e-8 * max(1.0, abs(psi[j])), (j, fd, psi[j])


def test_A_is_hessian_of_energy(orc):
    s = converged_tiny(orc)
    Q = np.zeros(s.n_ele)
    m = orc.A_modes(s.box, s.alpha, 1e-17)
    A = orc.build_A(s.box, s.eta, s.R, alpha_A=s.alpha)
    h = 0.05
    for (i, j) in [(0, 0), (3, 3), (0, 1), (2, 14), (5, 20)]:
        def U(di, dj):
            QQ = Q.copy()
            QQ[i] += di
            QQ[j] += dj
            return total_energy(orc, s, QQ, m)[0]
        if i == j:
            fd = (U(h, 0) - 2 * U(0, 0) + U(-h, 0)) / h ** 2
        else:
            fd = (U(h, h) - U(h, -h) - U(-h, h) + U(-h, -h)) / (4 * h * h)
        assert abs(fd - A[i, j]) < 1e-7 * abs(A).max(), (i, j, fd, A[i, j])


def test_forces_are_gradient_of_energy(orc):
    s = converged_tiny(orc)
    rng = np.random.default_rng(9)
    Q = rng.normal(scale=0.05, size=s.n_ele)
    Q -= Q.mean()
    m = orc.A_modes(s.box, s.alpha, 1e-17)
    _, ev = total_energy(orc, s, Q, m)
    F = ev["F_coul"] / orc.K_E
    h = 1e-5
    for i in range(s.n_ion):
        for d in range(3):
            sp, sm = copy.copy(s), copy.copy(s)
            sp.r = s.r.copy()
            sm.r = s.r.copy()
            sp.r[i, d] += h
            sm.r[i, d] -= h
            fd = -(total_energy(orc, sp, Q, m)[0] - total_energy(orc, sm, Q, m)[0]) / (2 * h)
            assert abs(fd - F[i, d]) < 1e-6 * np.abs(F).max() + 1e-8, (i, d, fd, F[i, d])


def test_alpha_independence(orc):
    """The Ewald split of Eq. 12 is exact: U, F and b do not depend on alpha."""
    rng = np.random.default_rng(3)
    out = []
    for alpha in (1.6, 2.4):
        s = converged_tiny(orc, alpha=alpha)
        if not out:
            Q = rng.normal(scale=0.1, size=s.n_ele)
            Q -= Q.mean()
        m = orc.A_modes(s.box, alpha, 1e-17)
        U, ev = total_energy(orc, s, Q, m)
        out.append((U, ev["F_coul"], full_b(orc, s, m)))
    (U1, F1, b1), (U2, F2, b2) = out
    assert abs(U1 - U2) < 1e-11 * abs(U1) + 1e-12
    assert np.abs(F1 - F2).max() < 1e-10 * np.abs(F1).max()
    assert np.abs(b1 - b2).max() < 1e-11 * np.abs(b1).max()


def test_A_alpha_dependence_is_background_only(orc):
    """Eq. 18 sums k != 0 only, so A carries the alpha-dependent neutralising-background
    constant: A(a) = A_0 + pi / (V a^2) e e^T, which drops out of e^T Q = 0.
    (The real-space sum runs over in-plane images only, so alpha (Lz - H) must be large enough
    that z-images are negligible: here Lz - H = 4 nm.)"""
    s = wl.one_shot_784()
    R = s.R[::6].copy()      # 64 sites over both walls
    a1, a2 = 1.6, 2.1
    A1 = orc.build_A(s.box, s.eta, R, alpha_A=a1)
    A2 = orc.build_A(s.box, s.eta, R, alpha_A=a2)
    V = s.box[0] * s.box[1] * s.box[2]
    shift = (math.pi / V) * (1 / a1 ** 2 - 1 / a2 ** 2)
    assert np.abs(A1 - A2 - shift).max() < 1e-12 * np.abs(A1).max()
    assert np.array_equal(A1, A1.T)
    assert np.linalg.eigvalsh(A1).min() > 0
    rng = np.random.default_rng(2)
    b = rng.normal(size=R.shape[0])
    side = s.side[::6]
    Q1, p1 = orc.cp_solve(orc.cho(A1), side, s.dpsi, b)
    Q2, p2 = orc.cp_solve(orc.cho(A2), side, s.dpsi, b)
    np.testing.assert_allclose(Q1, Q2, rtol=0, atol=1e-11 * np.abs(Q1).max())
    assert abs(p1 - p2) < 1e-11 * abs(p1)


def test_self_term_is_kernel_limit(orc):
    """2 (1/(sqrt(2 pi) eta) - alpha/sqrt(pi)) = lim_{R->0} [erfc(alpha R) - erfc(R/(sqrt 2 eta))]/R,
    so A_ij -> A_ii when R_j -> R_i (the k-space and slab terms are continuous)."""
    s = wl.tiny_slab()
    R = np.array([[0.3, 0.4, 0.5], [0.3 + 1e-5, 0.4, 0.5], [0.9, 0.1, s.H - 0.2]])
    A = orc.build_A(s.box, s.eta, R, alpha_A=1.7)
    assert abs(A[0, 1] - A[0, 0]) < 1e-6 * abs(A[0, 0])
    assert abs(A[0, 1] - A[1, 1]) < 1e-6 * abs(A[0, 0])


def q2d_far_energy(L, alpha, pos, w):
    """Far part of the exact quasi-2D energy, Eq. 14: a 2D lattice sum over (k_x, k_y) and an
    integral over k_z, done by adaptive quadrature (the integrand is even in k_z)."""
    kmax = 2 * alpha * math.sqrt(40.0)
    mx = int(kmax * L[0] / (2 * math.pi)) + 1
    my = int(kmax * L[1] / (2 * math.pi)) + 1
    tot = 0.0
    for a in range(-mx, mx + 1):
        for b in range(-my, my + 1):
            kx, ky = 2 * math.pi * a / L[0], 2 * math.pi * b / L[1]
            ph0 = kx * pos[:, 0] + ky * pos[:, 1]

            def f(kz):
                ph = ph0 + kz * pos[:, 2]
                s2 = (w @ np.cos(ph)) ** 2 + (w @ np.sin(ph)) ** 2
                k2 = kx * kx + ky * ky + kz * kz
                return 4 * math.pi / k2 * s2 * math.exp(-k2 / (4 * alpha * alpha))
            val, _ = scipy.integrate.quad(f, 1e-9, 2 * alpha * 7, epsabs=1e-13, epsrel=1e-12, limit=400)
            tot += 2 * val
    return tot / (4 * math.pi * L[0] * L[1])


@pytest.mark.slow
def test_slab_correction_converges_to_quasi2d(orc):
    """Eq. 16 + the slab term of Eq. 17 approach Eq. 14 as the vacuum gap Lz - H grows (§2,
    slab-correction paragraph).  alpha (Lz - H) >= 6 keeps the in-plane real-space sum exact."""
    base = converged_tiny(orc, alpha=4.0)
    rng = np.random.default_rng(11)
    Q = rng.normal(scale=0.1, size=base.n_ele)
    Q -= Q.mean()
    pos = np.concatenate([base.r, base.R])
    w = np.concatenate([base.q, Q])
    exact_far = q2d_far_energy(base.box, base.alpha, pos, w)
    errs = []
    for gap in (1.5, 2.25, 3.0):
        s = copy.copy(base)
        s.box = (base.box[0], base.box[1], base.H + gap)
        U, ev = total_energy(orc, s, Q)
        E = ev["E"] / orc.K_E
        # same real-space and self terms; compare the far parts: U_F + slab vs Eq. 14
        errs.append(abs((E[3] + E[5]) - exact_far))
    scale = abs(exact_far)
    assert errs[2] < 1e-5 * scale, (errs, scale)
    assert errs[1] < 0.2 * errs[0] and errs[2] < 0.2 * errs[1], errs


def test_cp_solution_neutral_and_equipotential(orc):
    s = wl.one_shot_784()
    sysm = orc.System(s, alpha_A=1.5)
    samples = orc.sample_metropolis(s.box, s.alpha, s.M, s.P, 3001, 0)
    m, c = sysm.modes(samples)
    ev = sysm.evaluate(m, c, with_lj=False)
    Q = ev["Q"]
    assert abs(Q.sum()) < 1e-13 * np.abs(Q).sum()
    psi = sysm.A @ Q - ev["b"]
    d = orc.potential_split(s.side)
    np.testing.assert_allclose(psi, ev["psi_bar"] + s.dpsi * d, rtol=0, atol=1e-10 * np.abs(psi).max())


def _mirror_sites(s):
    """index of the mirror image (z -> H - z) of every electrode site"""
    key = {(round(x, 9), round(y, 9), round(z, 9)): i for i, (x, y, z) in enumerate(s.R)}
    return np.array([key[(round(x, 9), round(y, 9), round(s.H - z, 9))] for x, y, z in s.R])


def test_mirror_antisymmetry(orc):
    """Mirror z -> H - z with q -> -q maps the problem onto itself with Q -> -Q (dpsi unchanged)."""
    s = wl.tiny_slab(n_pairs=2)
    half_r, half_q = s.r[:2].copy(), s.q[:2].copy()
    s.r = np.concatenate([half_r, half_r * [1, 1, -1] + [0, 0, s.H]])
    s.q = np.concatenate([half_q, -half_q])
    s.mol = np.arange(4, dtype=np.int32)
    s.itype = np.zeros(4, np.int32)
    s.mass = np.ones(4)
    mir = _mirror_sites(s)
    f = orc.cho(orc.build_A(s.box, s.eta, s.R, alpha_A=1.4))
    m = orc.A_modes(s.box, s.alpha, 1e-17)
    c = orc.ewald_weight(s.box, s.alpha, m)
    ev = orc.evaluate(s, f, m, c, with_lj=False)
    Q = ev["Q"]
    np.testing.assert_allclose(Q, -Q[mir], atol=1e-12 * np.abs(Q).max())
    # (psi_bar itself is not zero: the slab term ties the potential's zero to the z origin)


def test_empty_capacitor_parallel_plate(orc):
    """Sanity: an empty capacitor holds about dpsi * area / (4 pi d) per wall (Gaussian units)."""
    s = wl.one_shot_784()
    s.r, s.q = np.zeros((0, 3)), np.zeros(0)
    f = orc.cho(orc.build_A(s.box, s.eta, s.R, alpha_A=1.5))
    b = np.zeros(s.n_ele)
    Q, psibar = orc.cp_solve(f, s.side, s.dpsi, b)
    q_left = Q[s.side == 0].sum()
    est = -s.dpsi * s.box[0] * s.box[1] / (4 * math.pi * (s.H - 2 * wl.LAYER_DZ))
    assert q_left < 0
    assert 0.8 < q_left / est < 1.25, (q_left, est)
    mir = _mirror_sites(s)
    np.testing.assert_allclose(Q, -Q[mir], atol=1e-12 * np.abs(Q).max())


def test_lj_and_bond_forces_are_gradients(orc):
    """MD support terms (LJ 12-6 between ions of different molecules and ion-electrode, harmonic
    bonds): forces equal minus the finite-difference gradient of their energy."""
    s = wl.make_slab("lj", (1.6, 1.6, 9.0), 4, 4, 6, 3, alpha=2.0, eta_inv=10.0, rc=0.9, P=10, M=1,
                     seed=3, lam=3.0)
    s.lj_sigma = np.array([0.30, 0.28, 0.26, 0.32, 0.30])     # large enough to give real repulsion
    F, _, _ = orc.lj_bonds(s, s.r)

    def energy(r):
        _, e_lj, e_b = orc.lj_bonds(s, r)
        return e_lj + e_b
    h = 1e-6
    for i in range(0, s.n_ion, 3):
        for d in range(3):
            rp, rm = s.r.copy(), s.r.copy()
            rp[i, d] += h
            rm[i, d] -= h
            fd = -(energy(rp) - energy(rm)) / (2 * h)
            assert abs(fd - F[i, d]) < 1e-5 * np.abs(F).max() + 1e-6, (i, d, fd, F[i, d])


def test_sampled_evaluation_equals_rows_of_the_full_one(orc):
    """The subset evaluations used for checks at full size give the rows of the full evaluation."""
    from paper_2509_24742_gb300 import workloads as wl
    s = wl.one_shot_784()
    ref = orc.System(s, alpha_A=1.7)
    m, c = ref.modes(orc.sample_metropolis(s.box, s.alpha, s.M, s.P, 5, 0))
    ev = ref.evaluate(m, c, with_lj=False)
    t = np.array([0, 7, 399, 123, 250])
    Ft = orc.sampled_forces(s, m, c, ev["Q"], t)
    np.testing.assert_allclose(Ft, ev["F"][t], rtol=1e-13, atol=1e-12 * np.abs(ev["F"]).max())
    j = np.array([383, 0, 17, 200])
    np.testing.assert_allclose(orc.sampled_b(s, m, c, j), ev["b"][j], rtol=1e-13, atol=1e-13)


def test_A_rows_equal_rows_of_the_formed_A(orc):
    """The row evaluation used at sizes where A cannot be formed gives the rows of build_A times x."""
    from paper_2509_24742_gb300 import workloads as wl
    s = wl.tiny_slab(nx=3, ny=2)
    rng = np.random.default_rng(3)
    x = rng.normal(size=s.n_ele)
    A = orc.build_A(s.box, s.eta, s.R, 2.5)
    rows = np.array([0, 5, s.n_ele - 1])
    np.testing.assert_allclose(orc.A_rows(s.box, s.eta, s.R, 2.5, x, rows), (A @ x)[rows], rtol=1e-12,
                               atol=1e-12 * np.abs(A @ x).max())
