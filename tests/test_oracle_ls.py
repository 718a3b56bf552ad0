"""Pins of the oracle's per-pixel least-squares coefficients (Eq. (LS), Sec. II):
optimality over the window's guide values against the surrogate fit Eq. (11),
exactness when the centres are the guide's values, the constant guide, and a
literal normal-equation solve.  CPU only, small images."""
import numpy as np

from oracle import hdfilter_oracle as O


def _scene(seed, H=9, W=8, rho=3):
    rng = np.random.default_rng(seed)
    return rng.uniform(size=(rho, H, W)), rng.uniform(size=(2, H, W))


def _window_fit_residual(p, mu, sr, S, C):
    """sum over pixels of the (LS) objective for coefficients C (K, H, W)."""
    rho, H, W = p.shape
    total = 0.0
    for y in range(H):
        for x in range(W):
            th = p[:, max(0, y - S):y + S + 1, max(0, x - S):x + S + 1].reshape(rho, -1).T
            M = O.range_kernel(((th[:, None] - mu[None]) ** 2).sum(2), sr)
            t = O.range_kernel(((th - p[:, y, x]) ** 2).sum(1), sr)
            total += float(((M @ C[:, y, x] - t) ** 2).sum())
    return total


def test_ls_fits_the_window_at_least_as_well_as_the_surrogate():
    p, _ = _scene(1)
    mu, _, _ = O.bisecting_kmeans(p.reshape(3, -1).T, 4)
    C_ls = O.ls_coefficients(p, mu, 0.3, 2)
    C_opt = np.einsum("kl,lhw->khw", O.pinv_psd(O.kernel_matrix(mu, 0.3)), O.range_maps(p, mu, 0.3))
    r_ls = _window_fit_residual(p, mu, 0.3, 2, C_ls)
    r_opt = _window_fit_residual(p, mu, 0.3, 2, C_opt)
    assert r_ls <= r_opt * (1 + 1e-12)
    assert r_ls < 0.9 * r_opt   # strictly better on this scene


def test_ls_matches_the_normal_equations_where_full_rank():
    p, _ = _scene(2, H=7, W=7)
    mu, _, _ = O.bisecting_kmeans(p.reshape(3, -1).T, 3)
    C = O.ls_coefficients(p, mu, 0.4, 3)
    y, x = 3, 3                                     # a full 7 x 7 window
    th = p.reshape(3, -1).T
    M = O.range_kernel(((th[:, None] - mu[None]) ** 2).sum(2), 0.4)
    t = O.range_kernel(((th - p[:, y, x]) ** 2).sum(1), 0.4)
    c = np.linalg.solve(M.T @ M, M.T @ t)
    assert np.max(np.abs(C[:, y, x] - c)) <= 1e-8 * max(1.0, np.abs(c).max())


def test_ls_filter_is_exact_with_a_centre_per_value():
    rng = np.random.default_rng(3)
    vals = rng.uniform(size=(4, 3))
    lab = rng.integers(0, 4, size=(8, 9))
    lab.flat[:4] = np.arange(4)
    p = np.moveaxis(vals[lab], -1, 0)
    f = rng.uniform(size=(2, 8, 9))
    mu, _, _ = O.bisecting_kmeans(p.reshape(3, -1).T, 4)
    g = O.fast_filter(f, p, mu, 1.5, 0.3, 2, variant="ls")
    assert np.max(np.abs(g - O.bruteforce(f, p, 1.5, 0.3, 2))) <= 1e-10


def test_ls_constant_guide_returns_the_image_blur_ratio():
    p = np.full((3, 6, 7), 0.5)
    f = np.random.default_rng(4).uniform(size=(1, 6, 7))
    mu = np.array([[0.5, 0.5, 0.5]])
    g = O.fast_filter(f, p, mu, 1.0, 0.2, 2, variant="ls")
    assert np.max(np.abs(g - O.bruteforce(f, p, 1.0, 0.2, 2))) <= 1e-12
