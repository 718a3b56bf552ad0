"""Pins of the oracle's anisotropic range kernel (Sec. III-E: one sigma_r for
the low-light dimensions of the guide and another for the infrared one),
phi(x) = exp(-sum_d x_d^2 / (2 sigma_{r,d}^2)).  CPU only.

  - a two-pixel image whose filtered values follow by hand from Eq. (1)-(2);
  - one sigma_r repeated for every dimension gives the isotropic filter;
  - the anisotropic kernel of p is the unit isotropic kernel of the scaled
    guide p_d / sigma_{r,d};
  - K = number of distinct guide values makes Algorithm 1 equal the brute
    force (the exactness invariant, here with the anisotropic kernel);
  - the nearest centre of Eq. (17) is taken in the kernel's metric."""
import math

import numpy as np
import pytest

from oracle import hdfilter_oracle as O
from paper_1811_02363_gb300 import synthetic


def test_two_pixel_closed_form():
    # f = [0.2, 0.9] on a 1 x 2 image, guide p(0) = (0, 0), p(1) = (0.3, 0.1),
    # sigma_r = (0.5, 0.05), S = 1, sigma_s = 1.  Each pixel's window holds
    # itself (weight 1) and the other pixel at |j| = 1, of spatial weight
    # exp(-1/2) and range weight exp(-0.3^2 / (2 0.5^2) - 0.1^2 / (2 0.05^2))
    # = exp(-0.18 - 2.0); so w = exp(-2.68) and
    #   g(0) = (0.2 + 0.9 w) / (1 + w),  g(1) = (0.9 + 0.2 w) / (1 + w).
    f = np.array([[[0.2, 0.9]]])
    p = np.array([[[0.0, 0.3]], [[0.0, 0.1]]])
    w = math.exp(-2.68)
    want = np.array([(0.2 + 0.9 * w) / (1 + w), (0.9 + 0.2 * w) / (1 + w)])
    got = O.bruteforce(f, p, 1.0, [0.5, 0.05], 1)[0, 0]
    assert np.max(np.abs(got - want)) <= 1e-15
    got_at = O.bruteforce_at(f, p, 1.0, [0.5, 0.05], 1, np.array([[0, 0], [0, 1]]))[:, 0]
    assert np.max(np.abs(got_at - want)) <= 1e-15
    # the widths belong to their dimensions: swapped, the weight is exp(-0.5 - 18 - 0.02)
    w2 = math.exp(-0.5 - 0.09 / (2 * 0.05 ** 2) - 0.01 / (2 * 0.5 ** 2))
    got2 = O.bruteforce(f, p, 1.0, [0.05, 0.5], 1)[0, 0, 0]
    assert abs(got2 - (0.2 + 0.9 * w2) / (1 + w2)) <= 1e-15


def test_equal_widths_give_the_isotropic_filter():
    f = synthetic.color_rectangles(20, 17, seed=41)
    mu = O.bisecting_kmeans(f.reshape(3, -1).T.astype(np.float64), 5)[0]
    for fn in (lambda sr: O.bruteforce(f, f, 2.0, sr, 6),
               lambda sr: O.fast_filter(f, f, mu, 2.0, sr, 6),
               lambda sr: O.fast_filter(f, f, mu, 2.0, sr, 6, variant="indicator")):
        iso, ani = fn(0.2), fn([0.2, 0.2, 0.2])
        assert np.max(np.abs(iso - ani)) <= 1e-14
    pix = np.array([[0, 0], [7, 9], [19, 16]])
    a = O.fast_filter_at(f, f, mu, 2.0, 0.2, 6, pix)
    b = O.fast_filter_at(f, f, mu, 2.0, [0.2, 0.2, 0.2], 6, pix)
    assert np.max(np.abs(a - b)) <= 1e-14


def test_anisotropic_kernel_is_the_unit_kernel_of_the_scaled_guide():
    f = synthetic.color_rectangles(18, 21, seed=42)
    sr = np.array([0.1, 0.35, 0.2])
    q = O.scaled_guide(f, sr)
    assert np.allclose(q[1], f[1].astype(np.float64) / 0.35, rtol=0, atol=1e-15)
    a = O.bruteforce(f, f, 2.0, sr, 6)
    b = O.bruteforce(f, q, 2.0, 1.0, 6)
    assert np.max(np.abs(a - b)) <= 1e-13
    mu = O.bisecting_kmeans(q.reshape(3, -1).T, 6)[0]
    c = O.fast_filter(f, f, mu * sr[None, :], 2.0, sr, 6)
    d = O.fast_filter(f, q, mu, 2.0, 1.0, 6)
    assert np.max(np.abs(c - d)) <= 1e-10


def test_one_centre_per_distinct_value_equals_brute_force():
    rng = np.random.default_rng(43)
    vals = rng.uniform(0, 1, size=(5, 2))                      # 5 distinct guide values
    lab = rng.integers(0, 5, size=(12, 11))
    p = np.moveaxis(vals[lab], -1, 0)                          # (2, 12, 11)
    f = rng.uniform(0, 1, size=(1, 12, 11))
    sr = [0.15, 0.6]
    g = O.fast_filter(f, p, vals, 1.5, sr, 4)
    b = O.bruteforce(f, p, 1.5, sr, 4)
    assert np.max(np.abs(g - b)) <= 1e-10


def test_nearest_centre_in_the_kernels_metric():
    # centre 0 is nearer in plain distance, centre 1 in the scaled one
    mu = np.array([[0.0, 0.3], [0.3, 0.0]])
    p = np.array([[[0.1]], [[0.0]]])                            # (0.1, 0): plain d^2 0.1 vs 0.04
    assert O.nearest_center(p, mu)[0, 0] == 1
    # with sigma_r = (0.05, 1): scaled d^2 = 4 + 0.09 vs 16 -> centre 0
    assert O.nearest_center(p, mu, [0.05, 1.0])[0, 0] == 0
