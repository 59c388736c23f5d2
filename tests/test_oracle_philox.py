"""Pins for the oracle's random draws (Philox4x64-10 + Box-Muller).

The generator is pinned to numpy's independent Philox implementation (numpy's
bit generator increments its 256-bit counter before each block, so its block
for counter c is our block c + 1). The Gaussian transform is pinned to its
closed form at chosen points and to the N(0,1) law statistically.
"""
import math

import numpy as np
import pytest
from scipy import stats

from oracle import philox


@pytest.mark.parametrize("key", [(0, 0), (1, 0), (0xDEADBEEF12345678, 0x0123456789ABCDEF),
                                 (2 ** 64 - 1, 2 ** 64 - 1)])
@pytest.mark.parametrize("ctr", [(1, 0, 0, 0), (5, 7, 1, 2), (2 ** 40 + 3, 9, 0, 1),
                                 (17, 2 ** 63, 2 ** 64 - 1, 2)])
def test_philox4x64_matches_numpy(key, ctr):
    # explicit uint64 arrays: numpy converts Python int lists through float64
    ref = np.random.Philox(key=np.array(key, dtype=np.uint64),
                           counter=np.array([ctr[0] - 1, ctr[1], ctr[2], ctr[3]], dtype=np.uint64))
    want = ref.random_raw(4)
    got = philox.philox4x64_10(np.array([ctr], dtype=np.uint64), key)[0]
    assert [int(x) for x in got] == [int(x) for x in want]


def test_philox_counter_zero_numpy_first_block():
    # counter 0 of numpy (pre-increment) is our counter 1
    ref = np.random.Philox(key=np.array([123, 456], dtype=np.uint64), counter=0).random_raw(8)
    got = philox.philox4x64_10(np.array([[1, 0, 0, 0], [2, 0, 0, 0]], dtype=np.uint64), (123, 456))
    assert [int(x) for x in got.reshape(-1)] == [int(x) for x in ref]


def test_uniform_mapping_range():
    w = np.array([0, 2 ** 64 - 1, 2 ** 40 - 1, 2 ** 40], dtype=np.uint64)
    u = philox.uniforms24(w)
    assert u[0] == 0.5 * 2.0 ** -24
    assert u[1] == 1.0 - 0.5 * 2.0 ** -24
    assert u[2] == u[0]          # low 40 bits are dropped
    assert u[3] == 1.5 * 2.0 ** -24
    assert np.all((u > 0) & (u < 1))


def test_box_muller_closed_form():
    # u_a = e^{-1/2} gives radius 1; the angle 2 pi u_b picks the point on the circle
    ua = np.full(4, math.exp(-0.5))
    ub = np.array([0.0, 0.25, 0.5, 0.125])
    z0, z1 = philox.box_muller(ua, ub)
    np.testing.assert_allclose(z0, [1, 0, -1, math.sqrt(0.5)], atol=1e-15)
    np.testing.assert_allclose(z1, [0, 1, 0, math.sqrt(0.5)], atol=1e-15)
    # radius sqrt(-2 ln u)
    z0, z1 = philox.box_muller(np.array([0.1]), np.array([0.3]))
    assert math.isclose(math.hypot(z0[0], z1[0]), math.sqrt(-2 * math.log(0.1)), rel_tol=1e-14)


def test_normals_are_standard_normal():
    z = philox.normals(7, 3, 1, philox.TAG_G, 400_000)
    assert abs(z.mean()) < 0.01
    assert abs(z.var() - 1.0) < 0.01
    ks = stats.kstest(z, "norm")
    assert ks.pvalue > 1e-3
    # the two members of a Box-Muller pair and neighbouring pairs are uncorrelated
    zz = z.reshape(-1, 4)
    c = np.corrcoef(zz.T)
    assert np.max(np.abs(c - np.eye(4))) < 0.01


def test_streams_are_distinct_and_deterministic():
    a = philox.normals(1, 0, 0, philox.TAG_G, 64)
    assert np.array_equal(a, philox.normals(1, 0, 0, philox.TAG_G, 64))
    for other in [(2, 0, 0, 1), (1, 1, 0, 1), (1, 0, 1, 1), (1, 0, 0, 2)]:
        assert not np.allclose(a, philox.normals(*other, 64))
    # prefix property: the first k draws do not depend on how many are asked for
    assert np.array_equal(philox.normals(1, 0, 0, 1, 10), a[:10])


def test_gaussian_G_layout_and_sphere():
    G = philox.gaussian_G(5, 2, 1, 30, 7)
    flat = philox.normals(5, 2, 1, philox.TAG_G, 30 * 7)
    assert G.shape == (30, 7)
    assert G[3, 4] == flat[3 * 7 + 4]
    x = philox.sphere_x(5, 2, 1, 1000)
    assert math.isclose(np.linalg.norm(x), 1.0, rel_tol=1e-14)
