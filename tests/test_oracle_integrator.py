"""Pin of the oracle's integrator (Algorithm 1's MD step, oracle.System.md_step) by energy
conservation, independent of any GPU result.

With the thermostat off, velocity Verlet is symplectic and time-reversible, so over a fixed time the
error of the conserved quantity scales as dt^2.  Under constant potential the conserved quantity is
the Legendre transform of the energy in the electrode charges: H = KE + U(r, Q*) - dpsi d.Q*, where
Q* minimises U - dpsi d.Q on e^T Q = 0 (Eqs. 9-11).  Because Q* is a constrained minimiser,
dH/dr at fixed Q equals the total derivative, so the ion forces of Eq. 21 (Eq. 25 with every mode
kept) drive H exactly like a Hamiltonian.  The LJ potential is truncated at rc without a shift, so H
is evaluated with the shifted LJ energy (the truncated energy minus its value at rc for each pair
inside rc): that removes the jumps when pairs cross rc, while the force is unchanged.

A dropped half kick, a stale force in the second half kick, a missing mass, a z wrap or an x/y
wrap that moves a particle by anything but a box length each break the dt^2 law or the bound; the
last test plants one such mistake (the stale force) in a copy of the step and checks that the pin
catches it."""
import numpy as np
import pytest

from paper_2509_24742_gb300 import workloads as wl

ALPHA_A = 1.7
T_TOTAL = 0.1      # ps
DTS = (0.004, 0.002)


def _lj_shift(s, r):
    """Sum over LJ pairs inside rc of the truncated potential's value at rc, 4 eps ((sig/rc)^12 -
    (sig/rc)^6): ion-ion pairs of different molecules over every in-plane image, and ion-electrode
    pairs."""
    L = np.asarray(s.box, float)
    sig, eps = s.lj_tables()
    ele = sig.shape[0] - 1
    rc2 = s.rc * s.rc
    nimg = int(np.ceil(s.rc / min(L[0], L[1]))) + 1
    tot = 0.0
    for i in range(r.shape[0]):
        ti = s.itype[i]
        for ix in range(-nimg, nimg + 1):
            for iy in range(-nimg, nimg + 1):
                sh = np.array([ix * L[0], iy * L[1], 0.0])
                r2 = ((r[i] - r + sh) ** 2).sum(1)
                m = (r2 < rc2) & (r2 > 0) & (s.mol != s.mol[i])
                sr6 = (sig[ti, s.itype[m]] ** 2 / rc2) ** 3
                tot += 0.5 * (4.0 * eps[ti, s.itype[m]] * (sr6 * sr6 - sr6)).sum()
                ne = int((((r[i] - s.R + sh) ** 2).sum(1) < rc2).sum())
                sr6 = (sig[ti, ele] ** 2 / rc2) ** 3
                tot += ne * 4.0 * eps[ti, ele] * (sr6 * sr6 - sr6)
    return tot


def _hamiltonian(orc, s, r, v, ev):
    ke = 0.5 * float((s.mass[:, None] * v * v).sum())
    u = float(ev["E"].sum()) + ev.get("E_lj", 0.0) + ev.get("E_bond", 0.0)
    d = orc.potential_split(s.side)
    return ke + u - orc.K_E * s.dpsi * float(d @ ev["Q"]) - _lj_shift(s, r)


@pytest.fixture(scope="module")
def nve(orc):
    """24 ion sites (3-site cations with bonds, anions) between 2 x 16 x 3 electrode sites, every
    Fourier mode above 1e-10 kept, no thermostat.  The ions with the largest |v_x| and |v_y| start
    next to the x and y faces, moving out, so both periodic wraps happen during the run."""
    s = wl.make_slab("nve", (1.6, 1.6, 8.0), 4, 4, 6, 3, alpha=2.5, eta_inv=19.79, rc=1.6, P=0, M=0,
                     dpsi_volt=1.0, seed=5, with_md=True)
    L = np.asarray(s.box, float)
    for d in (0, 1):
        i = int(np.argmax(np.abs(s.v[:, d])))
        edge = L[d] - 1e-3 if s.v[i, d] > 0 else 1e-3
        s.r[:, d] = (s.r[:, d] + (edge - s.r[i, d])) % L[d]
    m = orc.full_modes(s.box, s.alpha, (20, 20, 80), tol=1e-10)
    c = orc.ewald_weight(s.box, s.alpha, m)
    return s, orc.System(s, alpha_A=ALPHA_A), m, c


def _run(orc, s, ref, m, c, dt, step_fn):
    s.dt = dt
    r, v = s.r.copy(), s.v.copy()
    ev = orc.evaluate(ref.at(r), ref.factor, m, c)
    F = ev["F"]
    h0 = _hamiltonian(orc, s, r, v, ev)
    dh, wraps = [], 0
    for _ in range(int(round(T_TOTAL / dt))):
        r_old = r
        r, v, ev = step_fn(r, v, F, m, c)
        F = ev["F"]
        wraps += int((np.abs(r[:, :2] - r_old[:, :2]) > 0.5 * np.asarray(s.box[:2])).sum())
        dh.append(_hamiltonian(orc, s, r, v, ev) - h0)
    return np.abs(dh).max(), wraps


def test_md_step_conserves_cp_hamiltonian_to_second_order(orc, nve):
    s, ref, m, c = nve
    e4, w4 = _run(orc, s, ref, m, c, DTS[0], ref.md_step)
    e2, w2 = _run(orc, s, ref, m, c, DTS[1], ref.md_step)
    ke = 0.5 * float((s.mass[:, None] * s.v ** 2).sum())
    print("max |H - H0| over %.2f ps: dt 4 fs %.3e, dt 2 fs %.3e kJ/mol (ratio %.3f; KE %.1f)"
          % (T_TOTAL, e4, e2, e4 / e2, ke))
    assert w4 >= 2 and w2 >= 2                # both the x and the y wrap were exercised
    assert 3.6 < e4 / e2 < 4.4                # second order in dt
    assert e2 < 1e-4 * ke


def test_planted_stale_force_breaks_the_pin(orc, nve):
    """A copy of md_step whose second half kick reuses the old force (a plausible slip) must fail."""
    s, ref, m, c = nve

    def stale(r, v, F, m_, c_):
        dt = s.dt
        v = v + 0.5 * dt * F / s.mass[:, None]
        r = r + dt * v
        r[:, 0] %= s.box[0]
        r[:, 1] %= s.box[1]
        ev = orc.evaluate(ref.at(r), ref.factor, m_, c_)
        v = v + 0.5 * dt * F / s.mass[:, None]
        return r, v, ev

    e4, _ = _run(orc, s, ref, m, c, DTS[0], stale)
    e2, _ = _run(orc, s, ref, m, c, DTS[1], stale)
    ke = 0.5 * float((s.mass[:, None] * s.v ** 2).sum())
    assert not (3.6 < e4 / e2 < 4.4 and e2 < 1e-4 * ke)
