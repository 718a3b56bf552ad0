"""Pins of the oracle's Young recursive Gaussian (the O(1) Gaussian
convolution Sec. II-C names): the library recursion against a literal loop,
unit gain, symmetry and closeness of the impulse response to a normalised
Gaussian, separability (rows and columns commute), Algorithm 1 with it
reducing to the normalised recursive blur when sigma_r is huge, the
coefficients against Young and van Vliet's published pole positions, and the
impulse response's variance against its closed form.  CPU only."""
import math

import numpy as np
import pytest

from oracle import hdfilter_oracle as O


def _loop(x, sigma):
    B, a1, a2, a3 = O.young_coefficients(sigma)
    L = len(x)
    w = np.zeros(L)
    for t in range(L):
        w[t] = B * x[t] + sum(a * w[t - i] for i, a in ((1, a1), (2, a2), (3, a3)) if t - i >= 0)
    y = np.zeros(L)
    for t in range(L - 1, -1, -1):
        y[t] = B * w[t] + sum(a * y[t + i] for i, a in ((1, a1), (2, a2), (3, a3)) if t + i < L)
    return y


@pytest.mark.parametrize("sigma", [0.8, 2.0, 5.0])
def test_recursion_matches_a_literal_loop(sigma):
    x = np.random.default_rng(1).uniform(-1, 1, size=40)
    assert np.max(np.abs(O.young_1d(x, sigma) - _loop(x, sigma))) <= 1e-12


def test_unit_gain_in_the_interior():
    # B = 1 - (a1 + a2 + a3): each pass keeps a constant, so far from the
    # borders a constant signal is returned unchanged
    for sigma in (1.0, 3.0, 8.0):
        y = O.young_1d(np.full(2000, 0.7), sigma)
        assert abs(y[1000] - 0.7) <= 1e-12
        B, a1, a2, a3 = O.young_coefficients(sigma)
        assert abs(B - (1 - a1 - a2 - a3)) <= 1e-15


@pytest.mark.parametrize("sigma,tol", [(2.0, 0.06), (5.0, 0.035), (8.0, 0.03)])
def test_impulse_response_is_a_symmetric_near_gaussian(sigma, tol):
    # the third-order recursion approximates the normalised Gaussian of
    # standard deviation sigma to a few per cent of its peak (closer for
    # larger sigma), with slightly heavier tails
    L, c = 1601, 800
    x = np.zeros(L)
    x[c] = 1.0
    h = O.young_1d(x, sigma)
    d = np.arange(1, 80)
    assert np.max(np.abs(h[c + d] - h[c - d])) <= 1e-12          # even response
    assert h.min() >= 0.0
    t = np.arange(L) - c
    g = np.exp(-t * t / (2 * sigma * sigma)) / (math.sqrt(2 * math.pi) * sigma)
    assert np.max(np.abs(h - g)) <= tol * g.max()
    assert abs(h.sum() - 1.0) <= 1e-9
    sd = math.sqrt(float((h * t * t).sum()))
    assert sigma <= sd <= 1.15 * sigma


def test_rows_and_columns_commute():
    x = np.random.default_rng(2).uniform(size=(2, 17, 23))
    a = O.young_1d(O.young_1d(x, 2.5, axis=-1), 2.5, axis=-2)
    b = O.young_1d(O.young_1d(x, 2.5, axis=-2), 2.5, axis=-1)
    assert np.max(np.abs(a - b)) <= 1e-13
    assert np.max(np.abs(O.spatial_conv(x, 2.5, 0, spatial="young") - a)) <= 1e-15


def test_fast_filter_with_huge_sigma_r_is_the_recursive_blur_ratio():
    rng = np.random.default_rng(3)
    f = rng.uniform(size=(2, 20, 18))
    mu = rng.uniform(size=(3, 2))
    g = O.fast_filter(f, f, mu, 2.0, 1e6, 0, spatial="young")
    one = O.spatial_conv(np.ones((20, 18)), 2.0, 0, spatial="young")
    ref = O.spatial_conv(f, 2.0, 0, spatial="young") / one
    assert np.max(np.abs(g - ref)) <= 1e-9


def test_planted_sign_error_is_caught():
    # the anticausal pass with the feedback sign flipped is far from the loop
    x = np.random.default_rng(4).uniform(size=30)
    B, a1, a2, a3 = O.young_coefficients(3.0)
    from scipy.signal import lfilter
    w = lfilter([B], [1.0, a1, a2, a3], x)
    wrong = np.flip(lfilter([B], [1.0, a1, a2, a3], np.flip(w)))
    assert np.max(np.abs(wrong - _loop(x, 3.0))) > 1e-2


# Young and van Vliet (1995) derive their recursion from the three poles of a
# rational approximation of the Gaussian's transfer function, at
# m0 = 1.16680 (real) and m1 +- i m2 = 1.10783 +- 1.40586 i, scaled by q: the
# causal pass has poles z = q / (m0 + q) and q / (m1 + q -+ i m2), i.e. its
# denominator is (m0 + q - q z^-1) ((m1 + q - q z^-1)^2 + m2^2) up to a
# constant factor.  Those pole positions are published numbers independent of
# the polynomial coefficients b0..b3 the oracle evaluates, so a digit dropped
# in any coefficient of b0..b3 moves the recursion off every pole product.
# The test finds the q whose pole product is closest to the oracle's
# normalised recursion (a1, a2, a3): the published coefficients are rounded
# to 5-6 digits, which leaves a best-fit residual below 3e-6 relative for
# 0.5 <= sigma <= 8; a dropped digit in any of them leaves 1.3e-5 or more at
# one of the sigmas below at least.
M0, M1, M2 = 1.16680, 1.10783, 1.40586


def _pole_product(q):
    poles = [q / (M0 + q), q / (M1 + q + 1j * M2), q / (M1 + q - 1j * M2)]
    return -np.real(np.poly(poles))[1:], poles   # a1, a2, a3 of w[t] = B x + sum a_i w[t-i]


@pytest.mark.parametrize("sigma", [0.6, 1.0, 2.0, 3.0, 5.0, 8.0])
def test_coefficients_are_the_published_pole_product(sigma):
    from scipy.optimize import minimize_scalar
    B, a1, a2, a3 = O.young_coefficients(sigma)
    got = np.array([a1, a2, a3])

    def resid(q):
        expect, _ = _pole_product(q)
        return float(np.max(np.abs(got - expect) / np.abs(expect)))

    fit = minimize_scalar(resid, bounds=(0.05, 50.0), method="bounded", options={"xatol": 1e-12})
    assert fit.fun <= 8e-6, fit.fun
    # the gain is the product of (1 - p_i) of the same poles (unit DC gain), up to
    # the coefficients' rounding carried through 1 - (a1 + a2 + a3)
    _, poles = _pole_product(fit.x)
    assert abs(B - float(np.real(np.prod([1 - p for p in poles])))) <= 1e-5 * (1 + np.abs(got).sum())


@pytest.mark.parametrize("sigma", [1.0, 3.0, 8.0])
def test_variance_of_the_impulse_response_has_the_closed_form(sigma):
    # a causal filter B / prod(1 - p_i z^-1) has an impulse response of
    # variance sum_i p_i / (1 - p_i)^2; the anticausal pass doubles it.
    B, a1, a2, a3 = O.young_coefficients(sigma)
    p = np.roots([1.0, -a1, -a2, -a3])
    var_closed = 2.0 * float(np.real(np.sum(p / (1.0 - p) ** 2)))
    L = 6000
    x = np.zeros(L)
    x[L // 2] = 1.0
    y = O.young_1d(x, sigma)
    t = np.arange(L) - L // 2
    var_num = float((y * t * t).sum() / y.sum())
    assert abs(var_num - var_closed) <= 1e-9 * var_closed
    # the recursion's spread tracks sigma (Young and van Vliet's design gives a
    # standard deviation a few to 25 per cent above sigma at these sizes)
    assert sigma ** 2 <= var_closed <= 1.6 * sigma ** 2
