"""Seeded synthetic inputs for the constant-potential slab workloads.

This module only places particles and assigns force-field constants; it holds
none of the electrostatics (no Ewald sums, no sampling law, no charge solve),
so both the CUDA path and the CPU oracle can take their inputs from it.

Geometry (a stand-in for the paper's graphene / coarse-grained ionic-liquid
supercapacitor of §4, whose force field is not reproduced here):

* The periodic box is ``Lx x Ly x Lz``; ``Lz`` is the Fourier period in z that
  already contains the vacuum padding (§2, the slab-correction paragraph after
  Eq. 17).  Walls and electrolyte occupy ``0 <= z <= H`` with ``H = Lz / lam``,
  lam = 1.5 unless stated.
* Each electrode is 3 layers of an ``nx x ny`` rectangular lattice, 0.335 nm
  apart: the left one at z = 0, 0.335, 0.67, the right one at H-0.67, H-0.335, H.
  Odd layers are shifted by half a lattice step in x.
* Ions are placed by random sequential addition (RSA) between the inner layers
  with a 0.3 nm gap to the walls, a minimum site-site distance ``d_min``, x/y
  periodic.  Cations are either point ions (``cation_sites=1``) or rigid
  triangles of side 0.35 nm with three +0.26 e sites; anions are -0.78 e points.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

K_E = 138.935458          # kJ mol^-1 nm e^-2 (Coulomb constant in MD units)
VOLT = 0.694461           # 1 V expressed as a potential in e/nm (96.4853 / K_E)
KB = 0.0083144626         # kJ mol^-1 K^-1

LAYER_DZ = 0.335
WALL_GAP = 0.3


@dataclass
class Slab:
    """All inputs of one constant-potential slab problem (units nm, ps, amu, e, kJ/mol)."""
    name: str
    box: tuple                      # (Lx, Ly, Lz), Lz = periodic length including vacuum
    H: float                        # wall-to-wall height
    alpha: float                    # Ewald splitting parameter, nm^-1
    eta: float                      # Gaussian width of the electrode charges (a length), nm
    rc: float                       # real-space cutoff, nm
    P: int                          # sampled Fourier modes per step
    M: int                          # deterministic modes (0,0,m_z), 1<=|m_z|<=M
    dpsi_volt: float                # right minus left electrode potential, V
    R: np.ndarray                   # electrode sites (n_ele, 3)
    side: np.ndarray                # int8 (n_ele,), 0 = left (negative for dpsi>0), 1 = right
    r: np.ndarray                   # ion sites (n_ion, 3)
    q: np.ndarray                   # ion charges (n_ion,)
    mol: np.ndarray                 # int32 molecule id per ion site
    itype: np.ndarray               # int32 LJ type per ion site
    mass: np.ndarray                # amu per ion site
    bonds: np.ndarray = field(default_factory=lambda: np.zeros((0, 2), np.int32))
    bond_r0: np.ndarray = field(default_factory=lambda: np.zeros(0))
    bond_k: float = 1000.0          # kJ mol^-1 nm^-2
    lj_sigma: np.ndarray = field(default_factory=lambda: np.zeros(0))   # per type; last type = electrode
    lj_eps: np.ndarray = field(default_factory=lambda: np.zeros(0))
    v: np.ndarray | None = None     # velocities (n_ion, 3), nm/ps
    dt: float = 0.002               # ps

    @property
    def n_ion(self):
        return int(self.r.shape[0])

    @property
    def n_ele(self):
        return int(self.R.shape[0])

    @property
    def dpsi(self):
        """Potential difference in e/nm (the unit of the Coulomb kernel 1/r)."""
        return self.dpsi_volt * VOLT

    def lj_tables(self):
        """Lorentz-Berthelot pair tables (sigma_ij, eps_ij), types x types."""
        s, e = np.asarray(self.lj_sigma, float), np.asarray(self.lj_eps, float)
        return 0.5 * (s[:, None] + s[None, :]), np.sqrt(e[:, None] * e[None, :])


def electrode_lattice(Lx, Ly, H, nx, ny, ax=None, ay=None):
    """3-layer walls at both ends of [0, H]; returns (R, side)."""
    ax = Lx / nx if ax is None else ax
    ay = Ly / ny if ay is None else ay
    zs_left = [0.0, LAYER_DZ, 2 * LAYER_DZ]
    zs_right = [H - 2 * LAYER_DZ, H - LAYER_DZ, H]
    R, side = [], []
    for s, zs in ((0, zs_left), (1, zs_right)):
        for li, z in enumerate(zs):
            shift = 0.5 * ax if (li % 2) else 0.0
            for iy in range(ny):
                for ix in range(nx):
                    R.append(((ix * ax + shift + 0.25 * ax) % Lx, (iy * ay + 0.25 * ay) % Ly, z))
                    side.append(s)
    return np.asarray(R, float), np.asarray(side, np.int8)


def _random_rotation(rng):
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


class _Grid:
    """Hash grid for the RSA overlap test (x, y periodic; z open)."""

    def __init__(self, Lx, Ly, cell):
        self.Lx, self.Ly = Lx, Ly
        self.nx, self.ny = max(1, int(Lx // cell)), max(1, int(Ly // cell))
        self.cx, self.cy, self.cz = Lx / self.nx, Ly / self.ny, cell
        self.cells = {}

    def key(self, p):
        return (int(p[0] // self.cx) % self.nx, int(p[1] // self.cy) % self.ny, int(math.floor(p[2] / self.cz)))

    def add(self, p):
        self.cells.setdefault(self.key(p), []).append(p)

    def clear(self, p, dmin2):
        kx, ky, kz = self.key(p)
        seen = set()
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                cxy = ((kx + dx) % self.nx, (ky + dy) % self.ny)
                for dz in (-1, 0, 1):
                    k = (cxy[0], cxy[1], kz + dz)
                    if k in seen:
                        continue
                    seen.add(k)
                    for o in self.cells.get(k, ()):
                        ddx = p[0] - o[0]
                        ddx -= self.Lx * round(ddx / self.Lx)
                        ddy = p[1] - o[1]
                        ddy -= self.Ly * round(ddy / self.Ly)
                        ddz = p[2] - o[2]
                        if ddx * ddx + ddy * ddy + ddz * ddz < dmin2:
                            return False
        return True


def place_electrolyte(rng, Lx, Ly, zlo, zhi, n_pairs, cation_sites, d_min, max_tries=2000):
    """RSA of n_pairs cations and n_pairs anions; returns (r, q, mol, kind) with kind 0..2 cation sites, 3 anion."""
    side_len = 0.35
    circ = side_len / math.sqrt(3.0)
    tri = np.array([[circ, 0.0, 0.0],
                    [-0.5 * circ, 0.5 * side_len, 0.0],
                    [-0.5 * circ, -0.5 * side_len, 0.0]])
    grid = _Grid(Lx, Ly, max(d_min, 1e-3))
    dmin2 = d_min * d_min
    r, q, mol, kind = [], [], [], []
    order = ["c"] * n_pairs + ["a"] * n_pairs      # bulky cations first: RSA jams later
    for mid, what in enumerate(order):
        for _ in range(max_tries):
            if what == "c" and cation_sites == 3:
                pad = circ
                c = np.array([rng.uniform(0, Lx), rng.uniform(0, Ly), rng.uniform(zlo + pad, zhi - pad)])
                sites = c + tri @ _random_rotation(rng).T
                sites[:, 0] %= Lx
                sites[:, 1] %= Ly
                qs, ks = [0.26, 0.26, 0.26], [0, 1, 2]
            else:
                sites = np.array([[rng.uniform(0, Lx), rng.uniform(0, Ly), rng.uniform(zlo, zhi)]])
                qs, ks = ([0.78], [0]) if what == "c" else ([-0.78], [3])
            if all(grid.clear(s, dmin2) for s in sites):
                for s, qq, kk in zip(sites, qs, ks):
                    grid.add(s)
                    r.append(s)
                    q.append(qq)
                    mol.append(mid)
                    kind.append(kk)
                break
        else:
            raise RuntimeError("RSA failed to place molecule %d (d_min=%.3f too large)" % (mid, d_min))
    return np.asarray(r), np.asarray(q), np.asarray(mol, np.int32), np.asarray(kind, np.int32)


def _rotations(u):
    """Rotation matrices from uniform triples (random unit quaternions, Shoemake's method)."""
    a = np.sqrt(1 - u[:, 0]) * np.sin(2 * np.pi * u[:, 1])
    b = np.sqrt(1 - u[:, 0]) * np.cos(2 * np.pi * u[:, 1])
    c = np.sqrt(u[:, 0]) * np.sin(2 * np.pi * u[:, 2])
    d = np.sqrt(u[:, 0]) * np.cos(2 * np.pi * u[:, 2])
    return np.stack([np.stack([1 - 2 * (c * c + d * d), 2 * (b * c - a * d), 2 * (b * d + a * c)], -1),
                     np.stack([2 * (b * c + a * d), 1 - 2 * (b * b + d * d), 2 * (c * d - a * b)], -1),
                     np.stack([2 * (b * d - a * c), 2 * (c * d + a * b), 1 - 2 * (b * b + c * c)], -1)], -2)


def place_electrolyte_lattice(rng, Lx, Ly, zlo, zhi, n_pairs, cation_sites, min_gap=0.08, rounds=50):
    """Fast placement for large replicas: one molecule per cell of a near-cubic grid filling the
    region (cells drawn at random when there are more cells than molecules), cation or anion at
    random, centre jittered by up to 15 % of the cell, triangles randomly rotated; molecules with a
    site closer than `min_gap` nm to a site of another molecule draw a new jitter and rotation
    (up to `rounds` times).  Returns (r, q, mol, kind, cell) like place_electrolyte plus the cell
    edge; neighbouring molecules start closer than in RSA, which the capped steepest-descent
    relaxation before MD removes."""
    from scipy.spatial import cKDTree
    n_mol = 2 * n_pairs
    h = zhi - zlo
    c = (Lx * Ly * h / n_mol) ** (1.0 / 3.0)
    nx, ny = max(1, int(Lx / c)), max(1, int(Ly / c))
    nz = max(1, int(math.ceil(n_mol / (nx * ny))))
    cx, cy, cz = Lx / nx, Ly / ny, h / nz
    cells = rng.permutation(nx * ny * nz)[:n_mol]
    ix, iy, iz = cells % nx, (cells // nx) % ny, cells // (nx * ny)
    base = np.c_[(ix + 0.5) * cx, (iy + 0.5) * cy, zlo + (iz + 0.5) * cz]
    is_cat = np.zeros(n_mol, bool)
    is_cat[rng.permutation(n_mol)[:n_pairs]] = True
    tri_mol = is_cat & (cation_sites == 3)
    nsite = np.where(tri_mol, 3, 1)
    first = np.concatenate([[0], np.cumsum(nsite)[:-1]])
    mol = np.repeat(np.arange(n_mol), nsite).astype(np.int32)
    kind = np.concatenate([[0, 1, 2] if t else ([0] if k else [3]) for t, k in zip(tri_mol, is_cat)]).astype(np.int32)
    q = np.where(kind == 3, -0.78, np.where(np.repeat(tri_mol, nsite), 0.26, 0.78))
    side_len = 0.35
    circ = side_len / math.sqrt(3.0)
    tri = np.array([[circ, 0.0, 0.0], [-0.5 * circ, 0.5 * side_len, 0.0], [-0.5 * circ, -0.5 * side_len, 0.0]])
    r = np.empty((int(nsite.sum()), 3))

    def draw(ms):
        centre = base[ms] + rng.uniform(-0.15, 0.15, size=(ms.size, 3)) * np.array([cx, cy, cz])
        rot = _rotations(rng.uniform(size=(ms.size, 3)))
        t3 = tri_mol[ms]
        pts = centre[t3][:, None, :] + np.einsum("sd,med->mse", tri, rot[t3])
        r[(first[ms[t3]][:, None] + np.arange(3)).ravel()] = pts.reshape(-1, 3)
        r[first[ms[~t3]]] = centre[~t3]
        idx = np.concatenate([(first[ms[t3]][:, None] + np.arange(3)).ravel(), first[ms[~t3]]])
        r[idx, 0] %= Lx
        r[idx, 1] %= Ly
        r[idx, 2] = np.clip(r[idx, 2], zlo, zhi)

    draw(np.arange(n_mol))
    for _ in range(rounds):
        tree = cKDTree(np.c_[r[:, :2], r[:, 2] - zlo + 1.0], boxsize=[Lx, Ly, 1e6])
        pairs = tree.query_pairs(min_gap, output_type="ndarray")
        if pairs.size:
            pairs = pairs[mol[pairs[:, 0]] != mol[pairs[:, 1]]]
        if not pairs.size:
            break
        draw(np.unique(mol[pairs[:, 1]]))
    return r, q, mol, kind, min(cx, cy, cz)


def maxwell_velocities(rng, mass, T):
    v = rng.normal(size=(mass.size, 3)) * np.sqrt(KB * T / mass)[:, None]
    v -= (mass[:, None] * v).sum(0) / mass.sum()
    return v


def _dmin_for_fraction(n_sites, volume, frac=0.3, cap=0.3):
    return min(cap, (frac * 6.0 * volume / (math.pi * n_sites)) ** (1.0 / 3.0))


def make_slab(name, box, nx, ny, n_pairs, cation_sites, *, alpha, eta_inv, rc, P, M=None,
              dpsi_volt=1.0, seed=0, ax=None, ay=None, T=400.0, with_md=False, lam=1.5, placement="rsa"):
    Lx, Ly, Lz = box
    H = Lz / lam
    rng = np.random.Generator(np.random.Philox(seed))
    R, side = electrode_lattice(Lx, Ly, H, nx, ny, ax, ay)
    zlo, zhi = 2 * LAYER_DZ + WALL_GAP, H - 2 * LAYER_DZ - WALL_GAP
    n_sites = n_pairs * (cation_sites + 1)
    if placement == "lattice":
        r, q, mol, kind, cell = place_electrolyte_lattice(rng, Lx, Ly, zlo, zhi, n_pairs, cation_sites)
        d_min = min(0.3, 0.8 * cell)
    else:
        # RSA of rigid triangles jams near 0.25 volume fraction; single sites fill to 0.3
        d_min = _dmin_for_fraction(n_sites, Lx * Ly * (zhi - zlo), frac=0.3 if cation_sites == 1 else 0.2)
        r, q, mol, kind = place_electrolyte(rng, Lx, Ly, zlo, zhi, n_pairs, cation_sites, d_min)
    if M is None:
        M = int(Lz // max(Lx, Ly))
    # types: 0..2 cation sites, 3 anion, 4 electrode; masses 67/42/15 and 145 amu
    masses = np.array([67.0, 42.0, 15.0, 145.0])
    if cation_sites == 1:
        masses[0] = 124.0
    mass = masses[kind]
    # LJ diameters 0.50/0.40/0.35 (cation sites), 0.45 (anion), 0.337 (electrode), scaled so that no
    # two RSA-placed ion sites start inside each other's repulsive core (sigma_max <= d_min); the
    # electrode diameter is kept, and the 0.3 nm wall gap stays outside sigma_ion-electrode
    sig = np.array([0.50, 0.40, 0.35, 0.45, 0.337])
    sig[:4] = sig[:4] * min(1.0, d_min / sig[:4].max())
    # eps 2 kJ/mol (ions) and 1 kJ/mol (electrode): with the scaled-down diameters a weaker
    # repulsion lets opposite charges collapse and the dense packing heat to thousands of K
    eps = np.array([2.0, 2.0, 2.0, 2.0, 1.0])
    bonds, r0 = np.zeros((0, 2), np.int32), np.zeros(0)
    if cation_sites == 3:
        b = []
        starts = np.flatnonzero(np.diff(np.concatenate([[-1], mol])) != 0)
        for s0 in starts:
            if kind[s0] == 0 and s0 + 2 < mol.size and mol[s0 + 2] == mol[s0]:
                b += [(s0, s0 + 1), (s0 + 1, s0 + 2), (s0, s0 + 2)]
        bonds = np.asarray(b, np.int32).reshape(-1, 2)
        r0 = np.full(bonds.shape[0], 0.35)
    v = maxwell_velocities(rng, mass, T) if with_md else None
    return Slab(name=name, box=(float(Lx), float(Ly), float(Lz)), H=H, alpha=alpha, eta=1.0 / eta_inv,
                rc=rc, P=P, M=M, dpsi_volt=dpsi_volt, R=R, side=side, r=r, q=q, mol=mol, itype=kind,
                mass=mass, bonds=bonds, bond_r0=r0, lj_sigma=sig, lj_eps=eps, v=v)


def one_shot_784(seed=1001):
    """Plain FP64 one-shot case: 2.0 x 2.0 x 12.0 nm, 2 x 3 layers of 8 x 8 sites at 0.246 nm,
    200 point cation/anion pairs, alpha 3.5, rc 1.2, eta^-1 19.79 nm^-1, P=100, M=2, 1 V."""
    return make_slab("slab784_P100", (2.0, 2.0, 12.0), 8, 8, 200, 1, alpha=3.5, eta_inv=19.79, rc=1.2,
                     P=100, M=2, dpsi_volt=1.0, seed=seed, ax=0.246, ay=0.246)


def md_11072(seed=1002):
    """MD case: 4.0 x 4.0 x 16.0 nm, 2 x 3 layers of 32 x 16 sites (3072), 2000 three-site cations and
    2000 anions (8000 ion sites), P=200, M=4, 1 V, 2 fs steps, Maxwell velocities at 400 K."""
    return make_slab("md11072_P200", (4.0, 4.0, 16.0), 32, 16, 2000, 3, alpha=3.5, eta_inv=19.79, rc=1.2,
                     P=200, M=4, dpsi_volt=1.0, seed=seed, with_md=True)


def precision_100k(seed=1003, dpsi_volt=2.0):
    """Precision-form case: 8 x 8 x 32 nm, 2 x 3 layers of 64 x 32 (12,288 sites), 21,928 cation/anion
    pairs (87,712 sites), P=500, 0-4 V.  alpha = 1.87 nm^-1 and rc = 1.6 nm, the paper's values for
    its own slab (§4): with alpha = 3.5 nm^-1 the sampled modes cover too small a share of this box's
    Fourier weight and the random-batch charge noise exceeds the charges tenfold.  Ions on the
    jittered grid (place_electrolyte_lattice): RSA at this size takes minutes."""
    return make_slab("prec100k_P500", (8.0, 8.0, 32.0), 64, 32, 21928, 3, alpha=1.87, eta_inv=19.79, rc=1.6,
                     P=500, M=4, dpsi_volt=dpsi_volt, seed=seed, with_md=True, placement="lattice")


def large_1m(seed=1006, dpsi_volt=2.0):
    """The 1.2 M-particle slab: 24 x 24 x 60 nm, 2 x 3 layers of 128 x 128 electrode sites (98,304),
    275,000 three-site cations and 275,000 anions (1.1 M ion sites), P = 1000, M = 2, 2 V.  alpha =
    1.2 nm^-1 with rc = 2.5 nm (alpha rc = 3, the paper's accuracy): at alpha 1.87 this box holds
    G ~ 40,000 effective modes and P = 1000 would leave the random-batch noise far above the
    forces; at 1.2, G / P ~ 11, as on the 11,072-site slab."""
    return make_slab("large1m_P1000", (24.0, 24.0, 60.0), 128, 128, 275000, 3, alpha=1.2, eta_inv=19.79, rc=2.5,
                     P=1000, M=None, dpsi_volt=dpsi_volt, seed=seed, with_md=True, placement="lattice")


def batch_replicas(n=64, seed=1004, n_total=(5000, 60000), sides=(16, 20, 24, 28, 32), aspect=(3.0, 8.0),
                   rho=50.0, P_range=(100, 400), alpha=1.87, rc=1.6):
    """Uneven replicas for the batching form: per replica an s x s lattice per layer at 0.25 nm
    (s from `sides`, so 1,536-6,144 electrode sites and Lx = Ly = s / 4 nm), a total particle count
    drawn from `n_total`, the electrolyte (3-site cations, 1-site anions) at `rho` sites per nm^3
    between the walls, Lz / Lx kept in `aspect` (the ion count follows when the aspect clamps),
    a voltage 0-4 V in 0.0625 V steps and a seed of its own.  P grows with the box volume V:
    50 ceil(V / 250 nm^3) clamped to `P_range` (a larger box spreads the same Fourier weight over
    more modes, and a fixed P would leave the charge noise growing with it).  alpha and rc are the
    paper's (§4).  Placement on a jittered grid (place_electrolyte_lattice) keeps generation fast at
    millions of sites."""
    rng = np.random.Generator(np.random.Philox(seed))
    out = []
    gap = 2 * (2 * LAYER_DZ + WALL_GAP)
    for i in range(n):
        s = int(sides[rng.integers(len(sides))])
        L = 0.25 * s
        ne = 6 * s * s
        sites = max(400.0, rng.uniform(*n_total) - ne)
        h = sites / (rho * L * L)
        a = min(max(1.5 * (h + gap) / L, aspect[0]), aspect[1])
        Lz = a * L
        h = Lz / 1.5 - gap
        n_pairs = max(50, int(rho * L * L * h / 4))
        P = int(min(P_range[1], max(P_range[0], 50 * math.ceil(L * L * Lz / 250.0))))
        dpsi = 0.0625 * int(rng.integers(0, 65))
        out.append(make_slab("replica%d_s%d_P%d" % (i, s, P), (L, L, Lz), s, s, n_pairs, 3, alpha=alpha,
                             eta_inv=19.79, rc=rc, P=P, M=None, dpsi_volt=dpsi, seed=seed * 1000 + i,
                             with_md=True, placement="lattice"))
    return out


def tiny_slab(seed=7, n_pairs=3, nx=2, ny=2, box=(1.2, 1.4, 9.0), alpha=2.0, rc=1.0, P=20, M=2,
              dpsi_volt=0.5, eta_inv=10.0, lam=3.0):
    """A few charges between two small walls (H = Lz / 3), for brute-force checks."""
    return make_slab("tiny", box, nx, ny, n_pairs, 1, alpha=alpha, eta_inv=eta_inv, rc=rc, P=P, M=M,
                     dpsi_volt=dpsi_volt, seed=seed, lam=lam)
