"""The oracle's Ewald sums against a published lattice constant.  A cubic box that holds one
conventional rock-salt cell (4 cations, 4 anions, a = 0.6 nm) is the infinite NaCl crystal as far as
the k-space sum (Eq. 16, periodic in z through L_z) is concerned.  With rc below the nearest-neighbour
distance r0 = a / 2 and alpha large enough that erfc(alpha r0) / r0 vanishes, the real-space sum is
empty, and the k-space and self terms must add up to the Madelung energy -4 M k_e q^2 / r0 of the
cell, whatever the origin; the slab term (Eq. 7's correction) must equal (2 pi / V) M_z^2 on its own,
zero when the origin makes M_z vanish.  A wrong normalisation of the mode weights, of the
exp(-k^2 / 4 alpha^2) factor or of the self term moves the result far outside the tolerance (the
real-space part is pinned by the gradient and alpha-independence tests)."""
import math
import os
from types import SimpleNamespace

import numpy as np

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "madelung_rock_salt.txt")


def madelung():
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            return float(line)
    raise ValueError("no value in " + GOLDEN)


def rock_salt(a, shift):
    frac = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5],
                     [0.5, 0, 0], [0, 0.5, 0], [0, 0, 0.5], [0.5, 0.5, 0.5]])
    r = (frac + shift) % 1.0 * a
    q = np.array([1.0] * 4 + [-1.0] * 4)
    return r, q


def test_ewald_energy_of_rock_salt_is_the_madelung_energy(orc):
    a, alpha, rc = 0.6, 26.0, 0.29
    M = madelung()
    V = a ** 3
    expect = -4.0 * M * orc.K_E / (a / 2)
    for shift in ([0.0, 0.0, 0.0], [0.13, 0.29, 0.07]):
        r, q = rock_salt(a, np.asarray(shift))
        # two uncharged electrode sites (the evaluation needs some; with Q = 0 they add nothing)
        R = np.array([[0.07, 0.11, 0.13], [0.37, 0.41, 0.43]])
        slab = SimpleNamespace(box=(a, a, a), r=r, q=q, R=R, alpha=alpha, eta=0.05, rc=rc,
                               side=np.array([0, 1], dtype=np.int8), dpsi=0.0, lj_sigma=np.zeros(0))
        m = orc.full_modes(slab.box, alpha, (44, 44, 44), tol=1e-30)
        c = orc.ewald_weight(np.asarray(slab.box), alpha, m)
        ev = orc.evaluate(slab, None, m, c, Q_fixed=np.zeros(2), with_lj=False)
        E = ev["E"]
        Mz = float((q * r[:, 2]).sum())
        assert E[0] == 0.0 and abs(E[1]) < 1e-12 and abs(E[2]) < 1e-12 and abs(ev["Mz"] - Mz) < 1e-12
        U = E[0] + E[3] + E[4]
        assert abs(U - expect) < 1e-9 * abs(expect), (shift, U, expect)
        assert abs(E[5] - 2.0 * math.pi / V * Mz * Mz * orc.K_E) <= 1e-12 * max(1.0, abs(E[5]))
