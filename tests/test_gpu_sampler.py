"""The exact sampler on the device (Eq. 26's P(k) by inverse CDF per dimension, rejection of I u {0}).

Integer work, so the bar is bit-exact: the device's modes equal the oracle's exact sampler and the
library's host sampler for the same (seed, step); the weights (Eqs. 24-25) equal the oracle's to
rounding; and an MD run whose captured steps sample on the device is bitwise the run that samples on
the host."""
import copy

import numpy as np
import pytest

from paper_2509_24742_gb300 import srbe, workloads as wl

pytestmark = pytest.mark.gpu
ALPHA_A = 1.7


@pytest.mark.parametrize("mmax", [(0, 0, 0), (8, 8, 48)])
def test_device_sampler_matches_host_and_oracle(orc, mmax):
    s = wl.one_shot_784()
    G = orc.G_closed(s.box, s.alpha, s.M, mmax)
    with srbe.from_slab(s, alpha_A=ALPHA_A) as c:
        c.set_sampler(srbe.EXACT, mmax)
        c.set_device_sampler(True)
        for seed, step in ((5, 0), (5, 1), (3002, 17), (2**40 + 3, 2**33 + 9)):
            m_dev, w_dev = c.sample_k_device(seed, step)
            c.sample_k(seed, step)
            m_host, _ = c.get_k()
            ref = orc.sample_exact(s.box, s.alpha, s.M, s.P, seed, step, mmax)
            assert np.array_equal(m_dev, m_host)
            assert np.array_equal(m_dev, ref)
            _, c_ref = orc.srbe_modes(s.box, s.alpha, s.M, ref, G)
            np.testing.assert_allclose(w_dev, c_ref[2 * s.M:], rtol=1e-14, atol=0)
    with srbe.from_slab(s, alpha_A=ALPHA_A) as c:
        with pytest.raises(srbe.SrbeError):
            c.set_device_sampler(True)        # the Metropolis sampler has no device form


def test_md_with_device_sampling_is_bitwise_host_sampling():
    s = wl.md_11072()
    out = []
    for dev in (False, True):
        with srbe.from_slab(s, precision=srbe.MIXED, md=True) as c:
            c.minimize(50)
            c.set_sampler(srbe.EXACT)
            if dev:
                c.set_device_sampler(True)
            c.step(12, 3002)
            assert c.graph_state()[0] == 1
            out.append(c.get_positions(velocities=True))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
