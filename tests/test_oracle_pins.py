"""Pins of the FP64 oracle against facts that do not come from the oracle:
hand-derived closed forms, literal brute force on tiny inputs, library
routines in the special cases where they coincide, and invariants the paper's
equations imply.  CPU only."""
import itertools
import math
import os

import numpy as np
import pytest
import scipy.ndimage
import scipy.signal

from oracle import hdfilter_oracle as O
from paper_1811_02363_gb300 import synthetic

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "closed_form_tiny.txt")


def _golden():
    rows = []
    for line in open(GOLDEN):
        if line.startswith("#") or not line.strip():
            continue
        name, y, x, val = line.split()
        rows.append((name, int(y), int(x), float(val)))
    return rows


TINY = {"A": np.array([[[0.0, 1.0, 0.0]]]), "B": np.array([[[0.0, 1.0], [1.0, 1.0]]])}


def _literal_bruteforce(f, p, sigma_s, sigma_r, S):
    """Eq. (1)-(2) with explicit loops over pixels and offsets."""
    n, H, W = f.shape
    g = np.zeros_like(f, dtype=np.float64)
    for y in range(H):
        for x in range(W):
            num = np.zeros(n)
            den = 0.0
            for j1 in range(-S, S + 1):
                for j2 in range(-S, S + 1):
                    qy, qx = y - j1, x - j2
                    if not (0 <= qy < H and 0 <= qx < W):
                        continue
                    w = math.exp(-(j1 * j1 + j2 * j2) / (2 * sigma_s ** 2))
                    d2 = sum((p[c, qy, qx] - p[c, y, x]) ** 2 for c in range(p.shape[0]))
                    wt = w * math.exp(-d2 / (2 * sigma_r ** 2))
                    num += wt * f[:, qy, qx]
                    den += wt
            g[:, y, x] = num / den
    return g


# ---------------------------------------------------------------- brute force

def test_bruteforce_closed_form_golden():
    for name, y, x, val in _golden():
        f = TINY[name]
        g = O.bruteforce(f, f, 1.0, 1.0, 1)
        assert abs(g[0, y, x] - val) < 1e-15


def test_bruteforce_matches_literal_loops():
    rng = np.random.default_rng(11)
    f = rng.uniform(size=(2, 6, 7))
    p = rng.uniform(size=(3, 6, 7))
    ref = _literal_bruteforce(f, p, 1.3, 0.4, 2)
    assert np.max(np.abs(O.bruteforce(f, p, 1.3, 0.4, 2) - ref)) < 1e-13
    pix = np.array([[0, 0], [5, 6], [2, 3]])
    at = O.bruteforce_at(f, p, 1.3, 0.4, 2, pix)
    assert np.max(np.abs(at - ref[:, pix[:, 0], pix[:, 1]].T)) < 1e-13


def test_bruteforce_constant_image_unchanged():
    f = np.full((3, 9, 8), 0.37)
    assert np.max(np.abs(O.bruteforce(f, f, 2.0, 0.1, 6) - f)) < 1e-15


def test_bruteforce_large_sigma_r_is_normalised_gaussian_blur():
    rng = np.random.default_rng(3)
    f = rng.uniform(size=(2, 12, 10))
    sigma_s, S = 1.5, 5
    t = np.arange(-S, S + 1)
    k2 = np.exp(-(t[:, None] ** 2 + t[None, :] ** 2) / (2 * sigma_s ** 2))
    num = np.stack([scipy.ndimage.correlate(c, k2, mode="constant") for c in f])
    den = scipy.ndimage.correlate(np.ones((12, 10)), k2, mode="constant")
    g = O.bruteforce(f, f, sigma_s, 1e8, S)
    assert np.max(np.abs(g - num / den)) < 1e-12


def test_bruteforce_tiny_sigma_r_distinct_guide_is_identity():
    rng = np.random.default_rng(4)
    H, W = 7, 6
    guide = rng.permutation(H * W).reshape(1, H, W) / 100.0     # distinct, spacing 0.01
    f = rng.uniform(size=(2, H, W))
    g = O.bruteforce(f, guide, 2.0, 1e-3, 3)
    assert np.max(np.abs(g - f)) < 1e-15


def test_bruteforce_linear_in_image_for_fixed_guide():
    rng = np.random.default_rng(5)
    p = rng.uniform(size=(3, 8, 9))
    f1, f2 = rng.uniform(size=(2, 2, 8, 9))
    g = lambda f: O.bruteforce(f, p, 1.0, 0.3, 3)
    assert np.max(np.abs(g(2.0 * f1 - 0.5 * f2) - (2.0 * g(f1) - 0.5 * g(f2)))) < 1e-13


# ---------------------------------------------------------------- convolution

def test_spatial_conv_separable_equals_direct_and_scipy():
    rng = np.random.default_rng(6)
    x = rng.normal(size=(2, 11, 13))
    sigma_s, S = 1.7, 6        # window wider than the image along one axis
    t = np.arange(-S, S + 1)
    k2 = np.exp(-(t[:, None] ** 2 + t[None, :] ** 2) / (2 * sigma_s ** 2))
    ref = np.stack([scipy.signal.convolve2d(c, k2, mode="same") for c in x])
    a = O.spatial_conv(x, sigma_s, S)
    b = O.spatial_conv_direct(x, sigma_s, S)
    assert np.max(np.abs(a - ref)) < 1e-12
    assert np.max(np.abs(b - ref)) < 1e-12


def test_spatial_conv_asymmetric_input_direction():
    # A single impulse must spread symmetrically (convolution with an even kernel).
    x = np.zeros((9, 9))
    x[2, 6] = 1.0
    out = O.spatial_conv(x, 1.0, 2)
    w = O.spatial_weights_1d(1.0, 2)
    for dy in range(-2, 3):
        for dx in range(-2, 3):
            assert abs(out[2 + dy, 6 + dx] - w[dy + 2] * w[dx + 2]) < 1e-15


# ---------------------------------------------------------------- pinv

@pytest.mark.parametrize("rank_deficient", [False, True])
def test_pinv_moore_penrose_conditions(rank_deficient):
    rng = np.random.default_rng(7)
    mu = rng.uniform(size=(6, 3))
    if rank_deficient:
        mu[4] = mu[1]              # duplicate centre -> singular Gram matrix
    A = O.kernel_matrix(mu, 0.5)
    X = O.pinv_psd(A)
    assert np.allclose(A @ X @ A, A, atol=1e-10)
    assert np.allclose(X @ A @ X, X, atol=1e-8 * max(1.0, np.abs(X).max()))
    assert np.allclose((A @ X).T, A @ X, atol=1e-10)
    assert np.allclose((X @ A).T, X @ A, atol=1e-10)
    assert np.allclose(X, np.linalg.pinv(A, hermitian=True), atol=1e-8 * max(1.0, np.abs(X).max()))
    if rank_deficient:
        assert np.linalg.matrix_rank(X) == 5


def test_kernel_matrix_unit_diagonal_symmetric():
    mu = np.random.default_rng(8).uniform(size=(5, 4))
    A = O.kernel_matrix(mu, 0.3)
    assert np.allclose(np.diag(A), 1.0) and np.allclose(A, A.T)
    assert abs(A[1, 3] - math.exp(-np.sum((mu[1] - mu[3]) ** 2) / (2 * 0.09))) < 1e-15


# ---------------------------------------------------------------- clustering

def test_bisecting_constant_data_single_cluster():
    P = np.full((50, 3), 0.25)
    mu, labels, sse = O.bisecting_kmeans(P, 8)
    assert mu.shape == (1, 3) and np.all(labels == 0) and sse[0] == 0.0


def test_bisecting_isolates_distinct_values():
    rng = np.random.default_rng(9)
    vals = rng.uniform(size=(6, 3)).astype(np.float32).astype(np.float64)
    P = vals[rng.integers(0, 6, size=400)]
    P[:6] = vals                                  # every value present
    mu, labels, sse = O.bisecting_kmeans(P, 6)
    assert mu.shape[0] == 6 and np.all(sse == 0.0)
    got = sorted(map(tuple, mu))
    assert np.allclose(np.array(got), np.array(sorted(map(tuple, vals))), atol=0)
    assert np.all(P == mu[labels])


def test_bisecting_split_order_and_convergence_by_replay():
    """Replay the greedy rule independently: at every step the cluster split
    is the one of largest SSE, and each split is a fixed point of Lloyd's
    2-means (every point nearer its own side's mean, ties to side a)."""
    rng = np.random.default_rng(10)
    P = np.concatenate([rng.normal(c, 0.05, size=(40, 2)) for c in
                        [(0, 0), (1, 0), (0, 1), (1, 1), (0.5, 0.5)]])
    P = P.astype(np.float32).astype(np.float64)
    members = [np.arange(len(P))]
    for K in range(2, 7):
        mu, labels, sse = O.bisecting_kmeans(P, K)
        prev_sse = [O.cluster_sse(P[m]) for m in members]
        c = int(np.argmax(prev_sse))
        # brute force: the new cluster K-1 is carved out of cluster c only
        assert set(np.where(labels == K - 1)[0]) | set(np.where(labels == c)[0]) == set(members[c])
        for k, m in enumerate(members):
            if k != c:
                assert set(np.where(labels == k)[0]) == set(m)
        a, b = members[c][labels[members[c]] == c], members[c][labels[members[c]] == K - 1]
        ma, mb = P[a].mean(0), P[b].mean(0)
        da = ((P[members[c]] - ma) ** 2).sum(1)
        db = ((P[members[c]] - mb) ** 2).sum(1)
        assert np.array_equal(db < da, labels[members[c]] == K - 1)
        members = [np.where(labels == k)[0] for k in range(K)]
        assert np.allclose(mu, np.stack([P[m].mean(0) for m in members]))


def test_clustering_error_decreases_with_K():
    P = synthetic.color_rectangles(32, 32, seed=1).reshape(3, -1).T.astype(np.float64)
    errs = []
    for K in (1, 2, 4, 8, 16):
        mu, labels, _ = O.bisecting_kmeans(P, K)
        errs.append(O.clustering_error(P, mu, labels))
    assert all(a >= b for a, b in zip(errs, errs[1:])) and errs[-1] < 0.5 * errs[0]


def test_nearest_center_ties_lowest_index():
    mu = np.array([[0.0], [1.0], [0.0]])
    p = np.array([[[0.5, 0.1, 0.9]]])
    assert list(O.nearest_center(p, mu)[0]) == [0, 0, 1]


# ---------------------------------------------------------------- fast filter

def test_fast_filter_closed_form_golden_with_two_clusters():
    # Two distinct guide values and K = 2: Algorithm 1 equals Eq. (1)-(2).
    for name, y, x, val in _golden():
        f = TINY[name]
        mu, _, _ = O.bisecting_kmeans(f.reshape(1, -1).T, 2)
        g = O.fast_filter(f, f, mu, 1.0, 1.0, 1)
        assert abs(g[0, y, x] - val) < 1e-14


def test_fast_filter_K_distinct_values_equals_bruteforce():
    rng = np.random.default_rng(12)
    vals = rng.uniform(size=(5, 3)).astype(np.float32).astype(np.float64)
    lab = rng.integers(0, 5, size=(14, 13))
    f = np.moveaxis(vals[lab], -1, 0)
    mu, _, _ = O.bisecting_kmeans(f.reshape(3, -1).T, 5)
    assert mu.shape[0] == 5
    g = O.fast_filter(f, f, mu, 2.0, 0.3, 6)
    assert np.max(np.abs(g - O.bruteforce(f, f, 2.0, 0.3, 6))) < 1e-12


def test_fast_filter_constant_image():
    f = np.full((3, 10, 11), 0.61)
    mu, _, _ = O.bisecting_kmeans(f.reshape(3, -1).T, 8)
    assert mu.shape[0] == 1
    assert np.max(np.abs(O.fast_filter(f, f, mu, 2.0, 0.2, 6) - f)) < 1e-14


def test_fast_filter_large_sigma_r_is_blur():
    rng = np.random.default_rng(13)
    f = rng.uniform(size=(2, 12, 14))
    mu = rng.uniform(size=(4, 2))
    A = O.kernel_matrix(mu, 1e8)
    assert np.allclose(A, 1.0)
    blur = O.spatial_conv(f, 1.5, 4) / O.spatial_conv(np.ones((12, 14)), 1.5, 4)
    g = O.fast_filter(f, f, mu, 1.5, 1e8, 4)
    assert np.max(np.abs(g - blur)) < 1e-12


def test_coefficients_are_unit_vectors_at_centres():
    rng = np.random.default_rng(14)
    mu = rng.uniform(size=(5, 3))
    A_pinv = O.pinv_psd(O.kernel_matrix(mu, 0.4))
    p = mu.T[:, :, None]                                   # pixels sitting on the centres
    B = O.range_maps(p, mu, 0.4)[:, :, 0]                  # (K, 5)
    assert np.allclose(A_pinv @ B, np.eye(5), atol=1e-10)


def test_fast_filter_invariant_to_centre_order_and_linear():
    f = synthetic.color_rectangles(20, 18, seed=2).astype(np.float64)
    mu, _, _ = O.bisecting_kmeans(f.reshape(3, -1).T, 6)
    g = O.fast_filter(f, f, mu, 2.0, 0.25, 6)
    perm = np.random.default_rng(0).permutation(6)
    assert np.max(np.abs(O.fast_filter(f, f, mu[perm], 2.0, 0.25, 6) - g)) < 1e-12
    f2 = np.random.default_rng(1).uniform(size=f.shape)
    lin = O.fast_filter(3 * f - f2, f, mu, 2.0, 0.25, 6)
    assert np.max(np.abs(lin - (3 * g - O.fast_filter(f2, f, mu, 2.0, 0.25, 6)))) < 1e-11


def test_fast_filter_at_matches_convolution_form():
    f = synthetic.hyperspectral_mixture(16, 15, bands=5, seed=3).astype(np.float64)
    mu, _, _ = O.bisecting_kmeans(f.reshape(5, -1).T, 7)
    g = O.fast_filter(f, f, mu, 1.5, 0.3, 5)
    pix = np.array([[0, 0], [15, 14], [7, 3], [3, 11]])
    at = O.fast_filter_at(f, f, mu, 1.5, 0.3, 5, pix)
    assert np.max(np.abs(at - g[:, pix[:, 0], pix[:, 1]].T)) < 1e-12


def test_psnr_improves_with_K():
    f = synthetic.color_rectangles(40, 40, seed=5).astype(np.float64)
    ref = O.bruteforce(f, f, 2.0, 0.2, 6)
    P = f.reshape(3, -1).T
    ps = []
    for K in (2, 8, 32):
        mu, _, _ = O.bisecting_kmeans(P, K)
        ps.append(O.psnr(O.fast_filter(f, f, mu, 2.0, 0.2, 6), ref))
    assert ps[0] < ps[1] < ps[2] and ps[2] > 35.0


def test_theorem1_bound_for_indicator_variant():
    f = synthetic.color_rectangles(24, 24, seed=6).astype(np.float64)
    sigma_s, sigma_r, S = 1.5, 0.2, 5
    g = O.bruteforce(f, f, sigma_s, sigma_r, S)
    L = math.exp(-0.5) / sigma_r                        # Lipschitz constant of phi
    Wn = (2 * S + 1) ** 2
    for K in (2, 4, 8):
        mu, _, _ = O.bisecting_kmeans(f.reshape(3, -1).T, K)
        gi = O.fast_filter(f, f, mu, sigma_s, sigma_r, S, variant="indicator")
        s = O.nearest_center(f, mu)
        E = float(((np.moveaxis(f, 0, -1) - mu[s]) ** 2).sum())
        assert ((gi - g) ** 2).sum() <= 4.0 * 3 * Wn ** 2 * L ** 2 * E


def test_guard_falls_back_to_indicator():
    # Centres chosen so that some coefficients go strongly negative; force
    # the guard by an absurd relative threshold and check the fallback value.
    f = synthetic.color_rectangles(12, 12, seed=7).astype(np.float64)
    mu = np.array([[0.2, 0.2, 0.2], [0.8, 0.8, 0.8], [0.5, 0.1, 0.9]])
    old = O.GUARD_REL
    try:
        O.GUARD_REL = 1e9
        g, st = O.fast_filter(f, f, mu, 1.0, 0.3, 3, return_stats=True)
    finally:
        O.GUARD_REL = old
    ind = O.fast_filter(f, f, mu, 1.0, 0.3, 3, variant="indicator", guard=False)
    assert st["fallback"] == 144 and np.max(np.abs(g - ind)) < 1e-14


# ---------------------------------------------------------------- NLM guide

def test_patch_vectors_and_pca_guide():
    f = synthetic.smooth_field_with_edges(20, 22, seed=1).astype(np.float64)
    X = O.patch_vectors(f, 5)
    assert X.shape == (25, 20, 22)
    assert np.array_equal(X[12], f[0])                      # patch centre
    assert X[0, 0, 0] == f[0, 2, 2]                         # mirrored corner (reflect, no repeat)
    guide, basis, lam = O.pca_guide(f, 5, 4)
    Xc = X.reshape(25, -1) - X.reshape(25, -1).mean(1, keepdims=True)
    ref_lam = np.linalg.svd(Xc / math.sqrt(Xc.shape[1]), compute_uv=False) ** 2
    assert np.allclose(lam, ref_lam, rtol=1e-9, atol=1e-12)
    assert np.allclose(guide.reshape(4, -1).var(axis=1), lam[:4], rtol=1e-9)
    assert np.allclose(basis @ basis.T, np.eye(4), atol=1e-12)


def test_psnr_definitions():
    a = np.zeros((3, 4, 5))
    b = np.full((3, 4, 5), 0.1)
    assert abs(O.psnr(a, b) - 20.0) < 1e-12
    assert abs(O.psnr_literal(a, b) - (20.0 - 10 * math.log10(3))) < 1e-12


def test_two_means_tie_goes_to_first_centre():
    # 1-D points 0, 0, 0.5, 1, 1: a = first point farthest from the mean (0),
    # b = 1; the middle point is equidistant (0.25 each) and goes to a; then
    # centre a = 1/6 keeps it.  Worked by hand.
    X = np.array([[0.0], [0.0], [0.5], [1.0], [1.0]])
    assert list(O.two_means_split(X)) == [False, False, False, True, True]


def test_pinv_keeps_small_but_significant_eigenvalues():
    # Nearly coincident centres: A is full rank with a tiny eigenvalue far
    # above MATLAB's default tolerance, so A^+ must be the true inverse.
    mu = np.array([[0.0, 0.0], [1e-3, 0.0], [0.5, 0.2]])
    A = O.kernel_matrix(mu, 1.0)
    lam = np.linalg.eigvalsh(A)
    assert lam.min() > 1e-9 and lam.min() < 1e-5
    X = O.pinv_psd(A)
    assert np.allclose(X @ A, np.eye(3), atol=1e-6)
