"""Pins of the oracle's random-batch part (§3, Eqs. 24-29, Theorems 3.1-3.2):

* Philox4x64-10 reproduces numpy's implementation of the same published generator;
* G of Eq. 27 in closed product form equals the brute lattice sum, and its
  continuum limit V alpha^3 / pi^(3/2);
* both samplers draw from P(k) of Eq. 26 (chi-square) and never from I u {0};
* SRBE b (Eq. 24) and force (Eq. 25) are unbiased estimators of the Ewald sums
  over the same lattice (Theorems 3.1 and 3.2: E xi = 0, E chi = 0), and their
  variance falls as 1/P;
* the deterministic low-|k_z| modes reduce the variance of b (Remark 3.1).
"""
import math

import numpy as np
import pytest
import scipy.stats

from paper_2509_24742_gb300 import workloads as wl


def test_philox_matches_numpy(orc):
    for key, ctr in [((0, 0), (0, 0, 0, 0)), ((123456789, 987654321), (5, 6, 7, 8)),
                     ((2 ** 64 - 1, 17), (2 ** 64 - 2, 2 ** 63, 1, 0))]:
        g = np.random.Philox(key=np.array(key, np.uint64), counter=np.array(ctr, np.uint64))
        ref = g.random_raw(4)            # numpy advances the counter by one before generating
        c1 = list(ctr)
        c1[0] = (c1[0] + 1) % 2 ** 64
        if c1[0] == 0:
            c1[1] = (c1[1] + 1) % 2 ** 64
        np.testing.assert_array_equal(orc.philox4x64(c1, key), ref)


@pytest.mark.parametrize("L,alpha,M,mmax", [((2.0, 2.0, 12.0), 3.5, 2, (0, 0, 0)),
                                            ((4.0, 4.0, 16.0), 3.5, 4, (0, 0, 0)),
                                            ((2.0, 2.0, 12.0), 3.5, 2, (8, 8, 48)),
                                            ((1.0, 1.2, 3.0), 2.5, 1, (2, 2, 6))])
def test_G_closed_form(orc, L, alpha, M, mmax):
    gc = orc.G_closed(L, alpha, M, mmax)
    gb = orc.G_brute(L, alpha, M, mmax)
    assert abs(gc - gb) < 1e-12 * gb
    if mmax == (0, 0, 0):
        cont = L[0] * L[1] * L[2] * alpha ** 3 / math.pi ** 1.5
        assert abs(gc / cont - 1) < 0.03


def _pk_table(L, alpha, M, mmax):
    cells, w = [], []
    for a in range(-mmax[0], mmax[0] + 1):
        for b in range(-mmax[1], mmax[1] + 1):
            for c in range(-mmax[2], mmax[2] + 1):
                if a == 0 and b == 0 and abs(c) <= M:
                    continue
                k2 = (2 * math.pi * a / L[0]) ** 2 + (2 * math.pi * b / L[1]) ** 2 + (2 * math.pi * c / L[2]) ** 2
                cells.append((a, b, c))
                w.append(math.exp(-k2 / (4 * alpha * alpha)))
    w = np.array(w)
    return {c: i for i, c in enumerate(cells)}, w / w.sum()


@pytest.mark.parametrize("kind", ["metropolis", "exact"])
def test_sampler_matches_target(orc, kind):
    L, alpha, M, mmax = (1.0, 1.2, 3.0), 2.5, 1, (2, 2, 6)
    idx, p = _pk_table(L, alpha, M, mmax)
    counts = np.zeros(p.size)
    fn = orc.sample_metropolis if kind == "metropolis" else orc.sample_exact
    for step in range(100):
        s = fn(L, alpha, M, 500, 77, step, mmax)
        for m in map(tuple, s):
            assert m in idx, m                      # never in I u {0}, never outside the box
            counts[idx[m]] += 1
    exp = p * counts.sum()
    keep = exp > 5
    chi2 = ((counts[keep] - exp[keep]) ** 2 / exp[keep]).sum()
    dof = keep.sum() - 1
    # chain states repeat on rejection; allow for the modest autocorrelation of the Metropolis chain
    infl = 1.5 if kind == "metropolis" else 1.0
    assert scipy.stats.chi2.sf(chi2 / infl, dof) > 1e-4, (chi2, dof)


def test_sampler_deterministic_and_unbounded(orc):
    L, alpha, M = (2.0, 2.0, 12.0), 3.5, 2
    a = orc.sample_metropolis(L, alpha, M, 100, 5, 9)
    b = orc.sample_metropolis(L, alpha, M, 100, 5, 9)
    c = orc.sample_metropolis(L, alpha, M, 100, 5, 10)
    assert np.array_equal(a, b) and not np.array_equal(a, c)
    assert not np.any((a[:, 0] == 0) & (a[:, 1] == 0) & (np.abs(a[:, 2]) <= M))


def _srbe_b_and_force(orc, s, G, mmax, P, seed, Q, step):
    samp = orc.sample_exact(s.box, s.alpha, s.M, P, seed, step, mmax)
    m, c = orc.srbe_modes(s.box, s.alpha, s.M, samp, G)
    S1 = orc.sfac(s.r, s.q, m, s.box)
    bF = orc.b_far(s.R, m, c, S1, s.box)
    S = S1 + orc.sfac(s.R, Q, m, s.box)
    kv = orc.kvectors(s.box, m)
    F = np.empty_like(s.r)
    orc.lib().orc_force_kspace(s.n_ion, orc._d(s.r), orc._d(s.q), kv.shape[0], kv, orc._d(c), orc._d(S), F)
    return bF, F


@pytest.mark.slow
def test_srbe_unbiased_and_variance_one_over_P(orc):
    """Theorems 3.1 / 3.2: E[b*_F] = b_F and E[F*] = F over the same (truncated) lattice,
    Var ~ 1/P.  The exact i.i.d. sampler and a lattice box shared with the Ewald sum make the
    expectation exact (the sampler's G is taken over the same box)."""
    s = wl.tiny_slab(alpha=2.0)
    mmax = (3, 3, 14)
    G = orc.G_closed(s.box, s.alpha, s.M, mmax)
    rng = np.random.default_rng(1)
    Q = rng.normal(scale=0.05, size=s.n_ele)
    Q -= Q.mean()
    m_full = orc.full_modes(s.box, s.alpha, mmax)
    c_full = orc.ewald_weight(s.box, s.alpha, m_full)
    S1 = orc.sfac(s.r, s.q, m_full, s.box)
    b_ref = orc.b_far(s.R, m_full, c_full, S1, s.box)
    S = S1 + orc.sfac(s.R, Q, m_full, s.box)
    kv = orc.kvectors(s.box, m_full)
    F_ref = np.empty_like(s.r)
    orc.lib().orc_force_kspace(s.n_ion, orc._d(s.r), orc._d(s.q), kv.shape[0], kv, c_full, orc._d(S), F_ref)
    var = {}
    for P in (8, 32):
        n = 3000
        bs, Fs = [], []
        for step in range(n):
            b, F = _srbe_b_and_force(orc, s, G, mmax, P, 1234 + P, Q, step)
            bs.append(b)
            Fs.append(F.ravel())
        bs, Fs = np.array(bs), np.array(Fs)
        zb = (bs.mean(0) - b_ref) / (bs.std(0, ddof=1) / math.sqrt(n))
        zf = (Fs.mean(0) - F_ref.ravel()) / (Fs.std(0, ddof=1) / math.sqrt(n))
        assert np.abs(zb).max() < 4.5, np.abs(zb).max()
        assert np.abs(zf).max() < 4.5, np.abs(zf).max()
        var[P] = (bs.var(0).mean(), Fs.var(0).mean())
    # quadrupling P divides the variance by 4 (within sampling error of ~10%)
    assert 3.2 < var[8][0] / var[32][0] < 4.8, var
    assert 3.2 < var[8][1] / var[32][1] < 4.8, var


def test_deterministic_modes_reduce_charge_variance(orc):
    """Remark 3.1: with M = 0 (plain RBE) the low-|k_z| modes are sampled and b is much noisier
    in an elongated cell; with M ~ Lz / max(Lx, Ly) the variance drops."""
    s = wl.one_shot_784()
    L = s.box
    out = {}
    for M in (0, 6):
        G = orc.G_closed(L, s.alpha, M)
        bs = []
        for step in range(150):
            samp = orc.sample_exact(L, s.alpha, M, 50, 99, step)
            m, c = orc.srbe_modes(L, s.alpha, M, samp, G)
            S1 = orc.sfac(s.r, s.q, m, L)
            bs.append(orc.b_far(s.R, m, c, S1, L))
        out[M] = np.array(bs).var(0).mean()
    assert out[6] < 0.5 * out[0], out
