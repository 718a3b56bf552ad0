"""Pins of the oracle's box spatial kernel (omega = 1 on W = [-S, S]^2, the
kernel Sec. III uses for nonlocal means), against things other than the
oracle itself: scipy's uniform filter, a literal loop over the definition
Eq. (1)-(2), closed forms and invariants.  CPU only."""
import math

import numpy as np
import pytest
from scipy import ndimage

from oracle import hdfilter_oracle as O


def _rng(seed):
    return np.random.default_rng(seed)


@pytest.mark.parametrize("S", [1, 2, 4])
def test_box_convolution_is_the_window_sum(S):
    # zero extension + unit weights: the sum over the clipped window, which
    # scipy's uniform filter (mean over the (2S+1)^2 window, zeros outside)
    # times the window size also computes
    x = _rng(1 + S).uniform(-1, 1, size=(2, 11, 13))
    got = O.spatial_conv(x, 1.0, S, spatial="box")
    ref = ndimage.uniform_filter(x, size=(1, 2 * S + 1, 2 * S + 1), mode="constant", cval=0.0)
    assert np.max(np.abs(got - ref * (2 * S + 1) ** 2)) <= 1e-12
    assert np.max(np.abs(O.spatial_conv_direct(x, 1.0, S, spatial="box") - got)) <= 1e-12


def test_box_impulse_response_is_the_window_indicator():
    x = np.zeros((1, 9, 9))
    x[0, 4, 4] = 1.0
    y = O.spatial_conv(x, 0.7, 2, spatial="box")[0]
    ind = np.zeros((9, 9))
    ind[2:7, 2:7] = 1.0
    assert np.array_equal(y, ind)


def _brute_loop(f, p, S, sr):
    """Eq. (1)-(2) with omega = 1, written as the literal quadruple loop."""
    n, H, W = f.shape
    g = np.zeros_like(f)
    for y in range(H):
        for x in range(W):
            num = np.zeros(n)
            den = 0.0
            for yy in range(max(0, y - S), min(H, y + S + 1)):
                for xx in range(max(0, x - S), min(W, x + S + 1)):
                    d2 = float(((p[:, yy, xx] - p[:, y, x]) ** 2).sum())
                    w = math.exp(-d2 / (2 * sr * sr))
                    num += w * f[:, yy, xx]
                    den += w
            g[:, y, x] = num / den
    return g


def test_box_bruteforce_matches_literal_loop():
    rng = _rng(7)
    f = rng.uniform(size=(2, 6, 7))
    p = rng.uniform(size=(3, 6, 7))
    got = O.bruteforce(f, p, 5.0, 0.3, 2, spatial="box")
    assert np.max(np.abs(got - _brute_loop(f, p, 2, 0.3))) <= 1e-13
    pix = np.array([[0, 0], [3, 4], [5, 6]])
    at = O.bruteforce_at(f, p, 5.0, 0.3, 2, pix, spatial="box")
    assert np.max(np.abs(at - got[:, pix[:, 0], pix[:, 1]].T)) <= 1e-13


def test_box_bruteforce_constant_and_flat_range_limits():
    f = np.full((3, 8, 9), 0.42)
    assert np.max(np.abs(O.bruteforce(f, f, 1.0, 0.2, 3, spatial="box") - 0.42)) <= 1e-15
    # sigma_r -> infinity: the normalised box blur (box * f) / (box * 1)
    rng = _rng(9)
    g = rng.uniform(size=(1, 10, 12))
    got = O.bruteforce(g, g, 1.0, 1e8, 2, spatial="box")
    ref = ndimage.uniform_filter(g[0], size=5, mode="constant") / \
        ndimage.uniform_filter(np.ones((10, 12)), size=5, mode="constant")
    assert np.max(np.abs(got[0] - ref)) <= 1e-9


def test_box_fast_filter_is_exact_with_a_centre_per_value():
    # K = number of distinct guide values: c(i) = e_s, Algorithm 1 equals the
    # brute force for any spatial kernel, the box included
    rng = _rng(11)
    vals = rng.uniform(size=(5, 3))
    lab = rng.integers(0, 5, size=(12, 10))
    lab.flat[:5] = np.arange(5)
    p = np.moveaxis(vals[lab], -1, 0)
    f = rng.uniform(size=(2, 12, 10))
    mu, _, _ = O.bisecting_kmeans(p.reshape(3, -1).T, 5)
    got = O.fast_filter(f, p, mu, 1.0, 0.25, 3, spatial="box")
    ref = O.bruteforce(f, p, 1.0, 0.25, 3, spatial="box")
    assert np.max(np.abs(got - ref)) <= 1e-11
    pix = np.array([[0, 0], [6, 5], [11, 9]])
    at = O.fast_filter_at(f, p, mu, 1.0, 0.25, 3, pix, spatial="box")
    assert np.max(np.abs(at - got[:, pix[:, 0], pix[:, 1]].T)) <= 1e-11


def test_planted_wrong_box_window_is_caught():
    # a box one tap too wide must fail the scipy pin
    x = _rng(3).uniform(size=(1, 9, 9))
    wrong = O.spatial_conv(x, 1.0, 3, spatial="box")
    ref = ndimage.uniform_filter(x, size=(1, 5, 5), mode="constant") * 25
    assert np.max(np.abs(wrong - ref)) > 1e-3
