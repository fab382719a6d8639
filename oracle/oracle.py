"""CPU oracle for SRBE constant-potential electrostatics (arXiv 2509.24742).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the CPU
baseline of ``bench.py`` call this; the library never does, and nothing here
imports the library.  The arithmetic lives in ``srbe_oracle.c`` (plain FP64
loops); this module loads it with ctypes and strings the steps together in the
order of Algorithm 1: sample -> b (Eq. 19 / Eq. 24) -> Q (Eqs. 9-11) ->
forces (Eq. 21 / Eq. 25 + Eq. 13 + slab term) -> integrate.

Units: nm, ps, amu, e, kJ/mol.  The C code works in Gaussian units (1/r); the
results are multiplied by the Coulomb constant K_E here.  Potentials (b, psi)
stay in e/nm: 1 V = 0.694461 e/nm.

Readings of the paper used here (also in the C file): slab term of A is
(4 pi/V) Z_i Z_j; slab term of b is -(4 pi Z_j/V) sum q_i z_i; b has no
"+ delta psi"; eta is a length; the Metropolis proposal width is
sigma_d = alpha L_d / (sqrt(2) pi).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np
import scipy.linalg

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "liboracle.so")
K_E = 138.935458
VOLT = 0.694461

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_up = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
_i64, _dbl, _int, _u64 = ctypes.c_int64, ctypes.c_double, ctypes.c_int, ctypes.c_uint64


def build(force=False):
    """Compile the oracle (gcc, OpenMP over independent output elements)."""
    src = os.path.join(HERE, "srbe_oracle.c")
    if not force and os.path.exists(LIB_PATH) and os.path.getmtime(LIB_PATH) >= os.path.getmtime(src):
        return LIB_PATH
    os.makedirs(os.path.dirname(LIB_PATH), exist_ok=True)
    tmp = LIB_PATH + ".tmp.%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11", "-o", tmp, src, "-lm"])
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB_PATH)
        L.orc_kvectors.argtypes = [_dp, _i64, _ip, _dp]
        L.orc_sfac.argtypes = [_i64, _dp, _dp, _i64, _dp, _dp]
        L.orc_b_far.argtypes = [_i64, _dp, _i64, _dp, _dp, _dp, _dp]
        L.orc_b_near.argtypes = [_dp, _dbl, _dbl, _dbl, _i64, _dp, _dp, _i64, _dp, _dp]
        L.orc_b_slab.argtypes = [_dp, _i64, _dp, _dp, _i64, _dp, _dp]
        L.orc_build_A.argtypes = [_dp, _dbl, _dbl, _dbl, _i64, _ip, _i64, _dp, _dp]
        L.orc_force_kspace.argtypes = [_i64, _dp, _dp, _i64, _dp, _dp, _dp, _dp]
        L.orc_dipole_z.argtypes = [_i64, _dp, _dp, _i64, _dp, _dp]
        L.orc_dipole_z.restype = _dbl
        L.orc_force_real.argtypes = [_dp, _dbl, _dbl, _dbl, _i64, _dp, _dp, _i64, _dp, _dp, _i64, ctypes.c_void_p,
                                     _dp, _dp]
        L.orc_energy_ee_real.argtypes = [_dp, _dbl, _dbl, _dbl, _i64, _dp, _dp]
        L.orc_energy_ee_real.restype = _dbl
        L.orc_force_lj.argtypes = [_dp, _dbl, _i64, _dp, _ip, _ip, _i64, _dp, ctypes.c_int32, ctypes.c_int32,
                                   _dp, _dp, _dp]
        L.orc_force_lj.restype = _dbl
        L.orc_force_bonds.argtypes = [_dp, _i64, _ip, _dp, _dbl, _dp, _dp]
        L.orc_force_bonds.restype = _dbl
        L.orc_philox4x64.argtypes = [_up, _up, _up]
        L.orc_sample_metropolis.argtypes = [_dp, _dbl, _int, _ip, _int, _u64, _u64, _ip]
        L.orc_sample_metropolis.restype = _i64
        L.orc_sample_exact.argtypes = [_dp, _dbl, _int, _ip, _int, _u64, _u64, _ip]
        L.orc_sample_exact.restype = _i64
        L.orc_G_brute.argtypes = [_dp, _dbl, _int, _ip]
        L.orc_G_brute.restype = _dbl
        L.orc_langevin_gauss.argtypes = [_u64, _u64, _i64, _dp]
        L.orc_A_rows.argtypes = [_dp, _dbl, _dbl, _dbl, _i64, _ip, _i64, _dp, _dp, _i64, ctypes.c_void_p, _dp]
        _lib = L
    return _lib


def _d(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a if shape is None else a.reshape(shape)


def _i(a):
    return np.ascontiguousarray(a, dtype=np.int32)


# ----------------------------------------------------------------------------- modes and weights
def kvectors(L, m):
    m = _i(m).reshape(-1, 3)
    kv = np.empty((m.shape[0], 3))
    lib().orc_kvectors(_d(L), m.shape[0], m, kv)
    return kv


def ewald_weight(L, alpha, m):
    """c_k = 4 pi exp(-k^2/4 alpha^2) / (V k^2), the per-mode factor of Eqs. 16, 18, 20, 21."""
    kv = kvectors(L, m)
    k2 = (kv ** 2).sum(1)
    V = L[0] * L[1] * L[2]
    return 4.0 * math.pi / (V * k2) * np.exp(-k2 / (4.0 * alpha * alpha))


def full_modes(L, alpha, mmax, tol=None):
    """Every nonzero m with |m_d| <= mmax_d (and exp(-k^2/4a^2) >= tol when tol is given)."""
    rng = [np.arange(-mm, mm + 1) for mm in mmax]
    g = np.stack(np.meshgrid(*rng, indexing="ij"), -1).reshape(-1, 3)
    g = g[np.any(g != 0, axis=1)]
    if tol is not None:
        k2 = ((2 * math.pi * g / np.asarray(L)) ** 2).sum(1)
        g = g[np.exp(-k2 / (4 * alpha * alpha)) >= tol]
    return _i(g)


def deterministic_modes(M):
    """The set I = {(0, 0, m_z): 1 <= |m_z| <= M} (after Eq. 25), both signs explicitly."""
    mz = [z for z in range(-M, M + 1) if z != 0]
    return _i([(0, 0, z) for z in mz]).reshape(-1, 3)


def G_closed(L, alpha, M, mmax=(0, 0, 0)):
    """G of Eq. 27 in product form: exp(-k^2/4a^2) factorises over dimensions, so
    G = theta_x theta_y theta_z - 1 - 2 sum_{m=1}^{M} exp(-pi^2 m^2 / (a L_z)^2)."""
    th = []
    for d in range(3):
        s = mmax[d] if mmax[d] > 0 else int(math.ceil(alpha * L[d] * math.sqrt(21 * math.log(10)) / math.pi))
        m = np.arange(-s, s + 1)
        th.append(np.exp(-(math.pi * m / (alpha * L[d])) ** 2).sum())
    mz_top = M if mmax[2] <= 0 else min(M, mmax[2])
    mz = np.arange(1, mz_top + 1)
    return th[0] * th[1] * th[2] - 1.0 - 2.0 * np.exp(-(math.pi * mz / (alpha * L[2])) ** 2).sum()


def G_brute(L, alpha, M, mmax=(0, 0, 0)):
    return lib().orc_G_brute(_d(L), alpha, M, _i(mmax))


def srbe_modes(L, alpha, M, samples, G):
    """Mode list and weights of Eqs. 24-25: the 2M deterministic modes with
    4 pi exp(-k^2/4a^2)/(V k^2) and each of the P samples with (G/P) 4 pi/(V k^2)."""
    det = deterministic_modes(M)
    samples = _i(samples).reshape(-1, 3)
    P = samples.shape[0]
    V = L[0] * L[1] * L[2]
    c_det = ewald_weight(L, alpha, det) if M > 0 else np.zeros(0)
    if P:
        k2 = (kvectors(L, samples) ** 2).sum(1)
        c_s = (G / P) * 4.0 * math.pi / (V * k2)
    else:
        c_s = np.zeros(0)
    return np.concatenate([det, samples]).astype(np.int32), np.concatenate([c_det, c_s])


def sample_metropolis(L, alpha, M, P, seed, step, mmax=(0, 0, 0)):
    out = np.empty((P, 3), np.int32)
    lib().orc_sample_metropolis(_d(L), alpha, M, _i(mmax), P, seed, step, out)
    return out


def sample_exact(L, alpha, M, P, seed, step, mmax=(0, 0, 0)):
    out = np.empty((P, 3), np.int32)
    lib().orc_sample_exact(_d(L), alpha, M, _i(mmax), P, seed, step, out)
    return out


def langevin_gauss(seed, step, n):
    """[n][3] standard normal numbers of the thermostat for step `step` (Philox4x64-10, Box-Muller)."""
    g = np.empty((int(n), 3))
    lib().orc_langevin_gauss(int(seed), int(step), int(n), g)
    return g


KB = 0.0083144626      # kJ mol^-1 K^-1


def langevin_o(v, mass, gamma, T, dt, seed, step):
    """Exact Ornstein-Uhlenbeck solution of the friction and noise terms of Eq. 39 over dt, with
    gamma read as a collision rate (1/ps): v <- e^{-gamma dt} v + sqrt((1 - e^{-2 gamma dt}) kB T / m) g."""
    if gamma <= 0.0:
        return v
    c1 = math.exp(-gamma * dt)
    sig = np.sqrt((1.0 - c1 * c1) * KB * T / np.asarray(mass, float))
    return c1 * v + sig[:, None] * langevin_gauss(seed, step, v.shape[0])


def philox4x64(ctr, key):
    out = np.empty(4, np.uint64)
    lib().orc_philox4x64(np.asarray(ctr, np.uint64), np.asarray(key, np.uint64), out)
    return out


# ----------------------------------------------------------------------------- building blocks
def sfac(pos, w, m, L):
    kv = kvectors(L, m)
    S = np.empty((kv.shape[0], 2))
    lib().orc_sfac(pos.shape[0], _d(pos), _d(w), kv.shape[0], kv, S)
    return S


def b_far(R, m, c, S1, L):
    kv = kvectors(L, m)
    out = np.empty(R.shape[0])
    lib().orc_b_far(R.shape[0], _d(R), kv.shape[0], kv, _d(c), _d(S1), out)
    return out


def b_near(L, alpha, eta, rc, r, q, R):
    out = np.empty(R.shape[0])
    lib().orc_b_near(_d(L), alpha, eta, rc, r.shape[0], _d(r), _d(q), R.shape[0], _d(R), out)
    return out


def b_slab(L, r, q, R):
    out = np.empty(R.shape[0])
    lib().orc_b_slab(_d(L), r.shape[0], _d(r), _d(q), R.shape[0], _d(R), out)
    return out


def A_modes(L, alpha_A, tol=1e-17):
    """Full lattice for A: every nonzero k with exp(-k^2 / 4 a^2) >= tol."""
    kmax = 2.0 * alpha_A * math.sqrt(-math.log(tol))
    mmax = [int(math.floor(kmax * L[d] / (2 * math.pi))) for d in range(3)]
    return full_modes(L, alpha_A, mmax, tol)


def A_rcut(alpha_A, tol=1e-17):
    """erfc(alpha r) < tol beyond this radius."""
    x = 1.0
    while math.erfc(x) >= tol:
        x += 0.01
    return x / alpha_A


def build_A(L, eta, R, alpha_A, tol=1e-17, modes=None, rcut=None):
    """Matrix A of Eq. 18 (Gaussian units, e/nm per e).  A does not depend on alpha_A
    beyond the truncation tolerance, so it is built with its own alpha_A."""
    m = A_modes(L, alpha_A, tol) if modes is None else _i(modes)
    rc = A_rcut(alpha_A, tol) if rcut is None else rcut
    n = R.shape[0]
    A = np.empty((n, n))
    lib().orc_build_A(_d(L), alpha_A, eta, rc, m.shape[0], m, n, _d(R), A)
    return A


def A_rows(L, eta, R, alpha_A, x, rows, tol=1e-17):
    """(A x)[rows] for the A of build_A, without forming A."""
    m = A_modes(L, alpha_A, tol)
    rc = A_rcut(alpha_A, tol)
    rws = np.ascontiguousarray(rows, dtype=np.int64)
    out = np.empty(rws.size)
    lib().orc_A_rows(_d(L), alpha_A, eta, rc, m.shape[0], m, R.shape[0], _d(R), _d(x), rws.size,
                     rws.ctypes.data_as(ctypes.c_void_p), out)
    return out


def potential_split(side):
    """d of Eq. 7: -1/2 on the left (negative) electrode, +1/2 on the right."""
    return np.where(np.asarray(side) == 0, -0.5, 0.5)


def cp_solve(factor, side, dpsi, b):
    """Charges under the neutrality constraint, Eqs. 9-11:
       psi_bar = - e^T A^-1 (dpsi d + b) / (e^T A^-1 e),  Q = J A^-1 (dpsi d + b),
       J = I - A^-1 e e^T / (e^T A^-1 e).   `factor` is scipy's Cholesky factor of A."""
    d = potential_split(side)
    e = np.ones(d.size)
    y = scipy.linalg.cho_solve(factor, dpsi * d + b)
    w = scipy.linalg.cho_solve(factor, e)
    psibar = -(e @ y) / (e @ w)
    Q = y - w * (e @ y) / (e @ w)
    return Q, psibar


def cho(A):
    return scipy.linalg.cho_factor(A, lower=True)


# ----------------------------------------------------------------------------- one evaluation
def evaluate(slab, factor, m, c, *, Q_fixed=None, with_lj=True):
    """One force + electrode-charge evaluation (Algorithm 1, lines 'compute b',
    'update Q', 'compute forces') for the weighted mode list (m, c).

    Returns a dict with b (e/nm), Q (e), psi_bar (e/nm), S1/S2 (complex [K]),
    F (kJ/mol/nm, Coulomb + optionally LJ/bonds), F_coul, and energy terms (kJ/mol):
    E = [U_N ion-ion, U_N ion-ele, U_N ele-ele, U_F, U_self, U_slab]."""
    L = np.asarray(slab.box, float)
    V = L[0] * L[1] * L[2]
    r, q, R = _d(slab.r), _d(slab.q), _d(slab.R)
    m = _i(m).reshape(-1, 3)
    c = _d(c)
    S1 = sfac(r, q, m, L)
    bF = b_far(R, m, c, S1, L)
    bN = b_near(L, slab.alpha, slab.eta, slab.rc, r, q, R)
    bS = b_slab(L, r, q, R)
    b = bF + bN + bS
    if Q_fixed is None:
        Q, psibar = cp_solve(factor, slab.side, slab.dpsi, b)
    else:
        Q, psibar = _d(Q_fixed), float("nan")
    S2 = sfac(R, Q, m, L)
    S = S1 + S2
    kv = kvectors(L, m)
    Fk = np.empty_like(r)
    lib().orc_force_kspace(r.shape[0], r, q, kv.shape[0], kv, c, _d(S), Fk)
    Mz = lib().orc_dipole_z(r.shape[0], r, q, R.shape[0], R, _d(Q))
    Fk[:, 2] += -(4.0 * math.pi / V) * q * Mz
    Fr = np.empty_like(r)
    Er = np.empty(2)
    lib().orc_force_real(L, slab.alpha, slab.eta, slab.rc, r.shape[0], r, q, R.shape[0], R, _d(Q), 0, None, Fr, Er)
    Eee = lib().orc_energy_ee_real(L, slab.alpha, slab.eta, slab.rc, R.shape[0], R, _d(Q))
    UF = 0.5 * float((c * (S ** 2).sum(1)).sum())
    Uself = (1.0 / (math.sqrt(2 * math.pi) * slab.eta) - slab.alpha / math.sqrt(math.pi)) * float(Q @ Q) \
        - slab.alpha / math.sqrt(math.pi) * float(q @ q)
    Uslab = 2.0 * math.pi / V * Mz * Mz
    F_coul = (Fk + Fr) * K_E
    out = dict(S1=S1[:, 0] + 1j * S1[:, 1], S2=S2[:, 0] + 1j * S2[:, 1], bF=bF, bN=bN, bS=bS, b=b, Q=Q,
               psi_bar=psibar, Mz=Mz, F_coul=F_coul, F_kspace=Fk * K_E, F_real=Fr * K_E,
               E=np.array([Er[0], Er[1], Eee, UF, Uself, Uslab]) * K_E)
    F = F_coul.copy()
    if with_lj and slab.lj_sigma.size:
        F_lj, E_lj, E_b = lj_bonds(slab, r)
        F += F_lj
        out.update(E_lj=E_lj, E_bond=E_b)
    out["F"] = F
    return out


def sampled_b(slab, m, c, sites):
    """b (e/nm, Eq. 24 with Eq. 19's near and slab parts) of the electrode sites `sites` only, from
    the structure factor of every ion: for checks at sizes where the full solve is out of reach."""
    L = np.asarray(slab.box, float)
    r, q = _d(slab.r), _d(slab.q)
    R = _d(np.asarray(slab.R)[np.asarray(sites)])
    m = _i(m).reshape(-1, 3)
    S1 = sfac(r, q, m, L)
    return b_far(R, m, _d(c), S1, L) + b_near(L, slab.alpha, slab.eta, slab.rc, r, q, R) + b_slab(L, r, q, R)


def sampled_forces(slab, m, c, Q, targets):
    """Electrostatic forces (kJ/mol/nm) on the ions `targets` only, for given electrode charges Q:
    k-space part of Eq. 25 with S = S1 + S2 over every particle, the slab term and the real-space
    pairs of Eq. 13 over every image within rc."""
    L = np.asarray(slab.box, float)
    V = L[0] * L[1] * L[2]
    r, q, R, Q = _d(slab.r), _d(slab.q), _d(slab.R), _d(Q)
    m = _i(m).reshape(-1, 3)
    c = _d(c)
    t = np.ascontiguousarray(targets, dtype=np.int64)
    S = sfac(r, q, m, L) + sfac(R, Q, m, L)
    kv = kvectors(L, m)
    rt, qt = _d(r[t]), _d(q[t])
    Fk = np.empty_like(rt)
    lib().orc_force_kspace(rt.shape[0], rt, qt, kv.shape[0], kv, c, _d(S), Fk)
    Mz = lib().orc_dipole_z(r.shape[0], r, q, R.shape[0], R, Q)
    Fk[:, 2] += -(4.0 * math.pi / V) * qt * Mz
    Fr = np.empty_like(rt)
    Er = np.empty(2)
    lib().orc_force_real(L, slab.alpha, slab.eta, slab.rc, r.shape[0], r, q, R.shape[0], R, Q, t.size,
                         t.ctypes.data_as(ctypes.c_void_p), Fr, Er)
    return (Fk + Fr) * K_E


def lj_bonds(slab, r):
    L = np.asarray(slab.box, float)
    sig, eps = slab.lj_tables()
    nt = sig.shape[0]
    F = np.zeros_like(r)
    e_lj = lib().orc_force_lj(L, slab.rc, r.shape[0], _d(r), _i(slab.mol), _i(slab.itype), slab.n_ele,
                              _d(slab.R), nt - 1, nt, _d(sig), _d(eps), F)
    Fb = np.zeros_like(r)
    e_b = 0.0
    if slab.bonds.shape[0]:
        e_b = lib().orc_force_bonds(L, slab.bonds.shape[0], _i(slab.bonds), _d(slab.bond_r0), slab.bond_k,
                                    _d(r), Fb)
    return F + Fb, e_lj, e_b


class System:
    """The oracle's view of one slab: A factored once (§2: A is constant), then
    evaluations for given mode lists."""

    def __init__(self, slab, alpha_A, tol=1e-17):
        self.slab = slab
        self.alpha_A = alpha_A
        self.A = build_A(slab.box, slab.eta, slab.R, alpha_A, tol)
        self.factor = cho(self.A)
        self.G = G_closed(slab.box, slab.alpha, slab.M)

    def modes(self, samples):
        return srbe_modes(self.slab.box, self.slab.alpha, self.slab.M, samples, self.G)

    def evaluate(self, m, c, **kw):
        return evaluate(self.slab, self.factor, m, c, **kw)

    def at(self, r):
        """A shallow copy of the slab with ion positions r."""
        import copy
        s2 = copy.copy(self.slab)
        s2.r = np.ascontiguousarray(r, dtype=np.float64)
        return s2

    def md_step(self, r, v, F, m, c, thermostat=None, step=0):
        """One step of Algorithm 1's integrator: half kick with F, drift, new SRBE forces at the new
        positions with the step's mode list (m, c), half kick (velocity Verlet); then, with
        thermostat = (gamma, T, seed), the Langevin friction and noise of Eq. 39 over the whole step
        (langevin_o with the noise of step `step`).  Electrode sites stay fixed; ions wrap in x and y.
        Returns (r, v, evaluation)."""
        s = self.slab
        dt = s.dt
        v = v + 0.5 * dt * F / s.mass[:, None]
        r = r + dt * v
        r[:, 0] %= s.box[0]
        r[:, 1] %= s.box[1]
        ev = evaluate(self.at(r), self.factor, m, c)
        v = v + 0.5 * dt * ev["F"] / s.mass[:, None]
        if thermostat is not None:
            gamma, T, seed = thermostat
            v = langevin_o(v, s.mass, gamma, T, dt, seed, step)
        return r, v, ev
