"""Thin Python binding of the SRBE C ABI (include/srbe.h): argument marshalling only.

Every computation happens in libsrbe.so (CUDA kernels for sm_103a).  There is no CPU fallback:
if the library cannot be built or loaded, or no GPU is present, the calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

SRBE_OK, SRBE_EINVAL, SRBE_ENOMEM, SRBE_ECUDA, SRBE_ESTATE, SRBE_ENOTCONV, SRBE_ETIMEOUT, SRBE_ENONFINITE = range(8)
FP64, MIXED = 0, 1
DIRECT, PCG, LATTICE = 0, 1, 2
WARM_ZERO, WARM_PREVIOUS, WARM_MODEL = 0, 1, 2
N_DESC = 80
METROPOLIS, EXACT = 0, 1
VOLT = 0.694461
K_E = 138.935458
ENERGY_TERMS = ("U_N ion-ion", "U_N ion-electrode", "U_N electrode-electrode", "U_F", "U_self", "U_slab",
                "U_LJ", "U_bond")

_STATUS = {SRBE_EINVAL: "invalid argument", SRBE_ENOMEM: "out of memory", SRBE_ECUDA: "CUDA error",
           SRBE_ESTATE: "call out of order", SRBE_ENOTCONV: "not converged", SRBE_ETIMEOUT: "timeout",
           SRBE_ENONFINITE: "non-finite result"}


class SrbeError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (_STATUS.get(code, "error"), code, msg))
        self.code = code


_lib = None
_vp, _dp, _i64, _int, _u64, _dbl = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int64, ctypes.c_int, \
    ctypes.c_uint64, ctypes.c_double
_ip = ctypes.POINTER(ctypes.c_int32)
_fp = ctypes.POINTER(ctypes.c_float)
_bp = ctypes.POINTER(ctypes.c_int8)

EXPORTS = {
    "srbe_create": ([_dp, _dbl, _dbl, _dbl, _int, _int, _dbl, _dbl, ctypes.POINTER(_vp)], _int),
    "srbe_destroy": ([_vp], _int),
    "srbe_last_error": ([_vp], ctypes.c_char_p),
    "srbe_set_stream": ([_vp, _vp], _int),
    "srbe_set_precision": ([_vp, _int], _int),
    "srbe_set_A_params": ([_vp, _dbl, _dbl], _int),
    "srbe_set_electrode": ([_vp, _i64, _dp, _bp], _int),
    "srbe_set_positions": ([_vp, _i64, _dp, _dp], _int),
    "srbe_get_positions": ([_vp, _dp, _dp], _int),
    "srbe_set_md": ([_vp, _dp, _dp, _int, _ip, _ip, _dp, _dp, _i64, _ip, _dp, _dbl, _dbl], _int),
    "srbe_set_sampler": ([_vp, _int, _ip], _int),
    "srbe_sample_k": ([_vp, _u64, _u64], _int),
    "srbe_set_device_sampler": ([_vp, _int], _int),
    "srbe_sample_k_device": ([_vp, _u64, _u64, _ip, _dp], _int),
    "srbe_get_k": ([_vp, _ip, _dp], _int),
    "srbe_set_k": ([_vp, _ip, _int], _int),
    "srbe_set_mode_list": ([_vp, _ip, _dp, _int], _int),
    "srbe_solve_electrode_charges": ([_vp, _dp, _dp, _dp], _int),
    "srbe_forces": ([_vp, _dp, _dp, _dp, _dp], _int),
    "srbe_step": ([_vp, _int, _u64], _int),
    "srbe_set_positions_dev": ([_vp, _i64, _vp, _vp], _int),
    "srbe_forces_dev": ([_vp, _vp, _vp], _int),
    "srbe_get_counters": ([_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64)], _int),
    "srbe_set_profiling": ([_vp, _int], _int),
    "srbe_set_graphs": ([_vp, _int], _int),
    "srbe_graph_state": ([_vp, ctypes.POINTER(_int), ctypes.POINTER(_i64)], _int),
    "srbe_get_phase_times": ([_vp, _dp, ctypes.POINTER(_i64)], _int),
    "srbe_structure_factor_noalloc": ([_dp, _i64, _vp, _vp, _int, _vp, _vp, _vp], _int),
    "srbe_synchronize": ([_vp, _dbl], _int),
    "srbe_set_host_io": ([_vp, _vp, _vp, _vp], _int),
    "srbe_forces_host_io": ([_vp, _u64, _u64, ctypes.POINTER(_dbl)], _int),
    "srbe_debug_inject_nonfinite": ([_vp, _int], _int),
    "srbe_minimize": ([_vp, _int, _dbl, _dbl, _u64], _int),
    "srbe_set_solver": ([_vp, _int, _dbl, _int, _int], _int),
    "srbe_get_solver_stats": ([_vp, ctypes.POINTER(_int), ctypes.POINTER(_dbl)], _int),
    "srbe_mlp_init": ([_vp, _u64], _int),
    "srbe_mlp_get_params": ([_vp, _fp, ctypes.POINTER(_i64)], _int),
    "srbe_mlp_set_params": ([_vp, _fp, _i64], _int),
    "srbe_descriptors": ([_vp, _fp], _int),
    "srbe_solution": ([_vp, _dp], _int),
    "srbe_mlp_predict": ([_vp, _fp, _i64, _fp], _int),
    "srbe_mlp_predict_dev": ([_vp, _vp, _i64, _vp], _int),
    "srbe_mlp_gradients": ([_vp, _fp, _fp, _i64, _fp, ctypes.POINTER(_dbl)], _int),
    "srbe_mlp_train": ([_vp, _fp, _fp, _i64, _int, _int, ctypes.c_float, ctypes.c_float, _u64,
                        ctypes.POINTER(_dbl)], _int),
    "srbe_charge_residual": ([_vp, _dp], _int),
    "srbe_set_thermostat": ([_vp, _dbl, _dbl, _u64], _int),
    "srbe_set_lattice": ([_vp, _int], _int),
    "srbe_lattice_info": ([_vp, _ip], _int),
    "srbe_set_skin": ([_vp, _dbl], _int),
    "srbe_get_skin": ([_vp], _dbl),
    "srbe_get_alpha_A": ([_vp], _dbl),
    "srbe_autotune_skin": ([_vp, _int, _u64, _dp, _int, _dp], _int),
    "srbe_autotune_tiles": ([_vp, _int, _u64, ctypes.POINTER(_int), _int, _dp], _int),
    "srbe_get_tiles": ([_vp], _int),
    "srbe_set_tiles": ([_vp, _int], _int),
    "srbe_batch_create": ([_int, ctypes.POINTER(_vp), ctypes.POINTER(_vp)], _int),
    "srbe_batch_destroy": ([_vp], _int),
    "srbe_batch_last_error": ([_vp], ctypes.c_char_p),
    "srbe_batch_set_width": ([_vp, _int], _int),
    "srbe_batch_get_width": ([_vp], _int),
    "srbe_batch_stream": ([_vp], _vp),
    "srbe_batch_step": ([_vp, _int, ctypes.POINTER(_u64), _dp], _int),
    "srbe_batch_autotune": ([_vp, _int, ctypes.POINTER(_u64), ctypes.POINTER(_int), _int, _dp], _int),
    "srbe_batch_autotune_tiles": ([_vp, _int, ctypes.POINTER(_u64), ctypes.POINTER(_int), _int, _dp], _int),
}
PHASES = ("upload", "cells", "S1", "rhs", "solve", "S2", "forces", "integrate", "energy", "forces_ii")


def library_path():
    return _build.LIB


def load(build=True):
    """Loads libsrbe.so (building it first when sources changed)."""
    global _lib
    if _lib is None:
        if build:
            _build.build()
        if not os.path.exists(_build.LIB):
            raise RuntimeError("libsrbe.so is missing; run paper_2509_24742_gb300.build.build()")
        L = ctypes.CDLL(_build.LIB)
        for name, (args, res) in EXPORTS.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _d(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None and a.size != n:
        raise ValueError("expected %d values, got %d" % (n, a.size))
    return a


def _ptr(a, t=_dp):
    return a.ctypes.data_as(t) if a is not None and a.size else None


class Context:
    """One SRBE problem on the GPU.  Units: nm, ps, amu, e, kJ/mol, V."""

    def __init__(self, box, alpha, eta, rc, P, M, psi_left=0.0, psi_right=1.0):
        self.lib = load()
        h = _vp()
        b = _d(box, 3)
        self._check(self.lib.srbe_create(_ptr(b), alpha, eta, rc, int(P), int(M), psi_left, psi_right,
                                         ctypes.byref(h)), None)
        self.h = h
        self.P, self.M = int(P), int(M)
        self.n_ion = 0
        self.n_ele = 0

    def _check(self, code, h="self"):
        if code != SRBE_OK:
            msg = self.lib.srbe_last_error(self.h if h == "self" else None)
            raise SrbeError(code, (msg or b"").decode())

    def close(self):
        if getattr(self, "h", None):
            self.lib.srbe_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # --- configuration
    def set_stream(self, stream_ptr):
        self._check(self.lib.srbe_set_stream(self.h, _vp(stream_ptr) if stream_ptr else None))

    def set_precision(self, mode):
        self._check(self.lib.srbe_set_precision(self.h, int(mode)))

    def set_A_params(self, alpha_A=0.0, tol=0.0):
        self._check(self.lib.srbe_set_A_params(self.h, float(alpha_A), float(tol)))

    def alpha_A(self):
        """The Ewald parameter A was built with."""
        return self.lib.srbe_get_alpha_A(self.h)

    def set_electrode(self, R, side):
        R = _d(R).reshape(-1, 3)
        side = np.ascontiguousarray(side, dtype=np.int8)
        self.n_ele = R.shape[0]
        self._check(self.lib.srbe_set_electrode(self.h, R.shape[0], _ptr(R), _ptr(side, _bp)))

    def set_positions(self, r, q):
        r = _d(r).reshape(-1, 3)
        q = _d(q, r.shape[0])
        self.n_ion = r.shape[0]
        self._check(self.lib.srbe_set_positions(self.h, r.shape[0], _ptr(r), _ptr(q)))

    def set_positions_dev(self, n, r_ptr, q_ptr):
        self.n_ion = int(n)
        self._check(self.lib.srbe_set_positions_dev(self.h, int(n), _vp(r_ptr), _vp(q_ptr)))

    def get_positions(self, velocities=False):
        r = np.empty((self.n_ion, 3))
        v = np.empty((self.n_ion, 3)) if velocities else None
        self._check(self.lib.srbe_get_positions(self.h, _ptr(r), _ptr(v) if velocities else None))
        return (r, v) if velocities else r

    def set_md(self, mass, itype, mol, lj_sigma, lj_eps, bonds=None, r0=None, kb=0.0, dt=0.002, v=None):
        n = self.n_ion
        mass = _d(mass, n)
        itype = np.ascontiguousarray(itype, dtype=np.int32)
        mol = np.ascontiguousarray(mol, dtype=np.int32)
        sig = _d(lj_sigma)
        eps = _d(lj_eps)
        nt = int(round(np.sqrt(sig.size)))
        bonds = np.zeros((0, 2), np.int32) if bonds is None else np.ascontiguousarray(bonds, dtype=np.int32)
        r0 = np.zeros(0) if r0 is None else _d(r0, bonds.shape[0])
        vv = None if v is None else _d(v, 3 * n)
        self._check(self.lib.srbe_set_md(self.h, _ptr(mass), _ptr(vv) if vv is not None else None, nt,
                                         _ptr(itype, _ip), _ptr(mol, _ip), _ptr(sig), _ptr(eps), bonds.shape[0],
                                         _ptr(bonds, _ip), _ptr(r0), float(kb), float(dt)))

    def set_sampler(self, kind=METROPOLIS, mmax=None):
        mm = None if mmax is None else np.ascontiguousarray(mmax, dtype=np.int32)
        self._check(self.lib.srbe_set_sampler(self.h, int(kind), _ptr(mm, _ip) if mm is not None else None))

    # --- modes
    def sample_k(self, seed, step=0):
        self._check(self.lib.srbe_sample_k(self.h, int(seed), int(step)))

    def set_device_sampler(self, on=True):
        self._check(self.lib.srbe_set_device_sampler(self.h, 1 if on else 0))

    def sample_k_device(self, seed, step=0):
        """The exact sampler's draw on the device: (m [P][3], w [P])."""
        m = np.empty((self.P, 3), np.int32)
        w = np.empty(self.P)
        self._check(self.lib.srbe_sample_k_device(self.h, int(seed), int(step), _ptr(m, _ip), _ptr(w)))
        return m, w

    def get_k(self):
        m = np.empty((self.P, 3), np.int32)
        G = ctypes.c_double()
        self._check(self.lib.srbe_get_k(self.h, _ptr(m, _ip), ctypes.byref(G)))
        return m, G.value

    def set_k(self, m):
        m = np.ascontiguousarray(m, dtype=np.int32).reshape(-1, 3)
        self.P = m.shape[0]
        self._check(self.lib.srbe_set_k(self.h, _ptr(m, _ip), m.shape[0]))

    def set_mode_list(self, m, w):
        m = np.ascontiguousarray(m, dtype=np.int32).reshape(-1, 3)
        w = _d(w, m.shape[0])
        self._check(self.lib.srbe_set_mode_list(self.h, _ptr(m, _ip), _ptr(w), m.shape[0]))

    # --- evaluation
    def solve_charges(self):
        Q = np.empty(self.n_ele)
        b = np.empty(self.n_ele)
        psi = ctypes.c_double()
        self._check(self.lib.srbe_solve_electrode_charges(self.h, _ptr(Q), ctypes.byref(psi), _ptr(b)))
        return Q, psi.value, b

    def forces(self, energy=False, out=None):
        """F (kJ/mol/nm), Q (e), psi_bar (V)[, energy terms].  `out=(F, Q)` writes into given
        C-contiguous float64 arrays (e.g. views of pinned host memory) instead of new ones."""
        if out is not None:
            F, Q = out
            assert F.dtype == np.float64 and F.flags.c_contiguous and F.size == 3 * self.n_ion
            assert Q.dtype == np.float64 and Q.flags.c_contiguous and Q.size == self.n_ele
        else:
            F = np.empty((self.n_ion, 3))
            Q = np.empty(self.n_ele)
        psi = ctypes.c_double()
        E = np.empty(8) if energy else None
        self._check(self.lib.srbe_forces(self.h, _ptr(F), _ptr(Q), ctypes.byref(psi),
                                         _ptr(E) if energy else None))
        return (F, Q, psi.value, E) if energy else (F, Q, psi.value)

    def forces_dev(self, F_ptr=None, Q_ptr=None):
        self._check(self.lib.srbe_forces_dev(self.h, _vp(F_ptr) if F_ptr else None, _vp(Q_ptr) if Q_ptr else None))

    def minimize(self, nsteps, a=2e-5, dmax=0.01, seed=9):
        self._check(self.lib.srbe_minimize(self.h, int(nsteps), float(a), float(dmax), int(seed)))

    def step(self, nsteps, seed0):
        self._check(self.lib.srbe_step(self.h, int(nsteps), int(seed0)))

    def set_host_io(self, r_ptr, F_ptr, Q_ptr=None):
        """Binds caller-owned page-locked host buffers (addresses): positions [n][3] in, forces
        [n][3] and charges [n_ele] out, all float64, for forces_host_io."""
        self._check(self.lib.srbe_set_host_io(self.h, _vp(r_ptr), _vp(F_ptr), _vp(Q_ptr) if Q_ptr else None))

    def forces_host_io(self, seed, step):
        """One captured force pass on the bound buffers; returns psi_bar (V)."""
        psi = _dbl()
        self._check(self.lib.srbe_forces_host_io(self.h, int(seed), int(step), ctypes.byref(psi)))
        return psi.value

    def synchronize(self, timeout_s=-1.0):
        """Waits for the queued work (at most timeout_s seconds; < 0 without limit) and reports the
        device-raised flags (SRBE_ENOTCONV, SRBE_ENONFINITE) as SrbeError; SRBE_ETIMEOUT at the limit."""
        self._check(self.lib.srbe_synchronize(self.h, float(timeout_s)))

    def debug_inject_nonfinite(self, what):
        """Test aid: 1 puts a NaN into F[0], 2 into Q[0] after every following pass, 0 stops it."""
        self._check(self.lib.srbe_debug_inject_nonfinite(self.h, int(what)))

    def set_graphs(self, on=True):
        self._check(self.lib.srbe_set_graphs(self.h, 1 if on else 0))

    def graph_state(self):
        """(1 live / 0 none / -1 capture failed, kernels per replayed step)."""
        cap, k = _int(), _i64()
        self._check(self.lib.srbe_graph_state(self.h, ctypes.byref(cap), ctypes.byref(k)))
        return cap.value, k.value

    def set_profiling(self, on=True):
        self._check(self.lib.srbe_set_profiling(self.h, 1 if on else 0))

    def phase_times(self):
        """{phase: (total ms, intervals)} since profiling was switched on."""
        ms = np.zeros(len(PHASES))
        cnt = (_i64 * len(PHASES))()
        self._check(self.lib.srbe_get_phase_times(self.h, _ptr(ms), cnt))
        return {p: (float(ms[i]), int(cnt[i])) for i, p in enumerate(PHASES)}

    # --- iterative solve and the learned warm start
    def set_solver(self, kind=PCG, tol=1e-8, maxit=1000, warm=WARM_ZERO):
        self._check(self.lib.srbe_set_solver(self.h, int(kind), float(tol), int(maxit), int(warm)))

    def solver_stats(self):
        it, res = _int(), _dbl()
        self._check(self.lib.srbe_get_solver_stats(self.h, ctypes.byref(it), ctypes.byref(res)))
        return it.value, res.value

    def mlp_init(self, seed=0):
        self._check(self.lib.srbe_mlp_init(self.h, int(seed)))

    def mlp_params(self):
        n = _i64()
        self._check(self.lib.srbe_mlp_get_params(self.h, None, ctypes.byref(n)))
        out = np.empty(n.value, np.float32)
        self._check(self.lib.srbe_mlp_get_params(self.h, _ptr(out, _fp), ctypes.byref(n)))
        return out

    def mlp_set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        self._check(self.lib.srbe_mlp_set_params(self.h, _ptr(p, _fp), p.size))

    def descriptors(self):
        D = np.empty((self.n_ele, N_DESC), np.float32)
        self._check(self.lib.srbe_descriptors(self.h, _ptr(D, _fp)))
        return D

    def solution(self):
        y = np.empty(self.n_ele)
        self._check(self.lib.srbe_solution(self.h, _ptr(y)))
        return y

    def mlp_predict(self, D):
        D = np.ascontiguousarray(D, dtype=np.float32).reshape(-1, N_DESC)
        out = np.empty(D.shape[0], np.float32)
        self._check(self.lib.srbe_mlp_predict(self.h, _ptr(D, _fp), D.shape[0], _ptr(out, _fp)))
        return out

    def mlp_predict_dev(self, D_ptr, n, out_ptr):
        """Forward pass on device buffers (float32 [n][80] -> float32 [n]), queued on the context's stream."""
        self._check(self.lib.srbe_mlp_predict_dev(self.h, _vp(D_ptr), int(n), _vp(out_ptr)))

    def mlp_gradients(self, D, T):
        D = np.ascontiguousarray(D, dtype=np.float32).reshape(-1, N_DESC)
        T = np.ascontiguousarray(T, dtype=np.float32).reshape(-1)
        n = self.mlp_params().size - 2 * N_DESC - 2
        g = np.empty(n, np.float32)
        loss = _dbl()
        self._check(self.lib.srbe_mlp_gradients(self.h, _ptr(D, _fp), _ptr(T, _fp), D.shape[0], _ptr(g, _fp),
                                                ctypes.byref(loss)))
        return g, loss.value

    def mlp_train(self, D, T, epochs=10, batch=512, lr=1e-3, weight_decay=1e-4, seed=0):
        D = np.ascontiguousarray(D, dtype=np.float32).reshape(-1, N_DESC)
        T = np.ascontiguousarray(T, dtype=np.float32).reshape(-1)
        loss = _dbl()
        self._check(self.lib.srbe_mlp_train(self.h, _ptr(D, _fp), _ptr(T, _fp), D.shape[0], int(epochs), int(batch),
                                            float(lr), float(weight_decay), int(seed), ctypes.byref(loss)))
        return loss.value

    def counters(self):
        a, b = _i64(), _i64()
        self._check(self.lib.srbe_get_counters(self.h, ctypes.byref(a), ctypes.byref(b)))
        return a.value, b.value

    def set_lattice(self, mode=1):
        """Lattice-electrode transforms: 0 never, 1 when N_ele x K is large (default), 2 always."""
        self._check(self.lib.srbe_set_lattice(self.h, int(mode)))

    def lattice_info(self):
        """(layers, nx, ny) of a recognised lattice electrode, else (0, 0, 0)."""
        d = np.zeros(3, np.int32)
        self._check(self.lib.srbe_lattice_info(self.h, d.ctypes.data_as(_ip)))
        return tuple(int(v) for v in d)

    def set_thermostat(self, gamma, T, seed=0):
        """Langevin thermostat of the MD step (gamma in 1/ps, 0 = off; T in K)."""
        self._check(self.lib.srbe_set_thermostat(self.h, float(gamma), float(T), int(seed)))

    def charge_residual(self):
        """FP64 relative residual of the constant-potential conditions met by the current charges."""
        r = _dbl()
        self._check(self.lib.srbe_charge_residual(self.h, ctypes.byref(r)))
        return r.value

    def set_skin(self, skin):
        self._check(self.lib.srbe_set_skin(self.h, float(skin)))

    def skin(self):
        return self.lib.srbe_get_skin(self.h)

    def autotune_skin(self, trial_steps, seed, skins=(0.05, 0.075, 0.1, 0.15, 0.2)):
        """Times each candidate Verlet skin, keeps the fastest; returns {skin: ms per step}."""
        sk = _d(skins)
        ms = np.zeros(sk.size)
        self._check(self.lib.srbe_autotune_skin(self.h, int(trial_steps), int(seed), _ptr(sk), sk.size, _ptr(ms)))
        return dict(zip(sk.tolist(), ms.tolist()))

    def autotune_tiles(self, trial_steps, seed, occ=(2, 4, 8, 16)):
        """Times each candidate structure-factor tile (blocks per SM its chunking keeps), keeps the
        fastest; returns {occ: ms per step}."""
        o = np.ascontiguousarray(occ, dtype=np.int32)
        ms = np.zeros(o.size)
        self._check(self.lib.srbe_autotune_tiles(self.h, int(trial_steps), int(seed),
                                                 o.ctypes.data_as(ctypes.POINTER(_int)), o.size, _ptr(ms)))
        return dict(zip(o.tolist(), ms.tolist()))

    def tiles(self):
        return self.lib.srbe_get_tiles(self.h)

    def set_tiles(self, occ):
        """Blocks per SM the structure factor's particle chunking keeps (1..64, default 8)."""
        self._check(self.lib.srbe_set_tiles(self.h, int(occ)))


class Batch:
    """Many replicas (Contexts) stepped as one CUDA graph launch per step; the contexts are borrowed
    and must outlive the batch."""

    def __init__(self, contexts):
        self.lib = load()
        self.ctxs = list(contexts)
        arr = (_vp * len(self.ctxs))(*[c.h for c in self.ctxs])
        h = _vp()
        code = self.lib.srbe_batch_create(len(self.ctxs), arr, ctypes.byref(h))
        if code != SRBE_OK:
            raise SrbeError(code, "srbe_batch_create failed")
        self.h = h

    def _check(self, code):
        if code != SRBE_OK:
            raise SrbeError(code, (self.lib.srbe_batch_last_error(self.h) or b"").decode())

    def _seeds(self, seeds):
        s = np.ascontiguousarray(seeds, dtype=np.uint64)
        if s.size != len(self.ctxs):
            raise ValueError("one seed per replica")
        return s, s.ctypes.data_as(ctypes.POINTER(_u64))

    def close(self):
        if getattr(self, "h", None):
            self.lib.srbe_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_width(self, width):
        self._check(self.lib.srbe_batch_set_width(self.h, int(width)))

    def width(self):
        return self.lib.srbe_batch_get_width(self.h)

    def stream(self):
        """The batch's cudaStream_t as an integer (for torch.cuda.ExternalStream)."""
        return self.lib.srbe_batch_stream(self.h) or 0

    def step(self, nsteps, seeds, residuals=False):
        """nsteps steps of every replica; with residuals=True returns each replica's FP64 check."""
        s, sp = self._seeds(seeds)
        res = np.zeros(len(self.ctxs)) if residuals else None
        self._check(self.lib.srbe_batch_step(self.h, int(nsteps), sp, _ptr(res) if residuals else None))
        return res

    def autotune(self, trial_steps, seeds, widths=None):
        """Times each candidate stream width, keeps the fastest; returns {width: ms per batch step}."""
        n = len(self.ctxs)
        if widths is None:
            widths = sorted({0, 1, 2, 4, 8, 16, 32, n} & set(range(n + 1)))
        w = np.ascontiguousarray(widths, dtype=np.int32)
        ms = np.zeros(w.size)
        s, sp = self._seeds(seeds)
        self._check(self.lib.srbe_batch_autotune(self.h, int(trial_steps), sp,
                                                 w.ctypes.data_as(ctypes.POINTER(_int)), w.size, _ptr(ms)))
        return dict(zip(w.tolist(), ms.tolist()))

    def autotune_tiles(self, trial_steps, seeds, occ=(2, 4, 8, 16)):
        """Times each candidate structure-factor tile for every replica at once, keeps the fastest;
        returns {occ: ms per batch step}."""
        o = np.ascontiguousarray(occ, dtype=np.int32)
        ms = np.zeros(o.size)
        s, sp = self._seeds(seeds)
        self._check(self.lib.srbe_batch_autotune_tiles(self.h, int(trial_steps), sp,
                                                       o.ctypes.data_as(ctypes.POINTER(_int)), o.size, _ptr(ms)))
        return dict(zip(o.tolist(), ms.tolist()))


def structure_factor_noalloc(box, n, r_ptr, w_ptr, K, m_ptr, S_ptr, stream_ptr=None):
    """S(k) for caller-owned device buffers (r [n][3], w [n], m [K][3] int32, S [K][2]) without
    any device allocation by the library; see include/srbe.h for the limits."""
    L = load()
    b = _d(box, 3)
    code = L.srbe_structure_factor_noalloc(_ptr(b), int(n), _vp(r_ptr), _vp(w_ptr), int(K), _vp(m_ptr),
                                           _vp(S_ptr), _vp(stream_ptr) if stream_ptr else None)
    if code != SRBE_OK:
        raise SrbeError(code, "srbe_structure_factor_noalloc failed")


def from_slab(slab, precision=FP64, alpha_A=0.0, md=False):
    """Convenience: a Context set up from a workloads.Slab (electrode, positions, optionally MD terms)."""
    ctx = Context(slab.box, slab.alpha, slab.eta, slab.rc, slab.P, slab.M, 0.0, slab.dpsi_volt)
    ctx.set_precision(precision)
    ctx.set_A_params(alpha_A, 0.0)
    ctx.set_electrode(slab.R, slab.side)
    ctx.set_positions(slab.r, slab.q)
    if md:
        sig, eps = slab.lj_tables()
        ctx.set_md(slab.mass, slab.itype, slab.mol, sig, eps, slab.bonds, slab.bond_r0, slab.bond_k, slab.dt,
                   v=slab.v if slab.v is not None else np.zeros((slab.n_ion, 3)))
    return ctx
