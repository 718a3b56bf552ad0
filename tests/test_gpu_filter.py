"""GPU parity of the filter path against the FP64 oracle, element by element.

The CUDA path gets the oracle's centres (rounded to float32, which both sides
then use), so that clustering differences cannot leak into the filter
comparison.  Tolerance for float32 paths: max-abs <= 1e-4."""
import numpy as np
import pytest
import torch

from oracle import hdfilter_oracle as O
from paper_1811_02363_gb300 import synthetic

pytestmark = pytest.mark.gpu
TOL = 1e-4


@pytest.fixture(scope="module")
def api():
    from paper_1811_02363_gb300 import build
    build.build()
    from paper_1811_02363_gb300 import api as A
    assert torch.cuda.is_available()
    return A


def _cuda(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def _centres(p, K):
    mu, _, _ = O.bisecting_kmeans(p.reshape(p.shape[0], -1).T.astype(np.float64), K)
    return mu.astype(np.float32)


CASES = [
    # name, image maker, separate guide?, K, sigma_s, sigma_r
    ("rgb_150x97_S9", lambda: synthetic.color_rectangles(150, 97, seed=21), False, 8, 3.0, 0.2),
    ("rgb_70x200_S15", lambda: synthetic.color_rectangles(70, 200, seed=22), False, 12, 5.0, 0.25),
    ("hyper31_80x70_S15", lambda: synthetic.hyperspectral_mixture(80, 70, 31, seed=23), False, 32, 5.0, 0.3),
    ("rgb_100x90_S24", lambda: synthetic.color_rectangles(100, 90, seed=24), False, 16, 8.0, 0.15),
    ("gray_guide6_96x130_S15", lambda: synthetic.smooth_field_with_edges(96, 130, seed=25), True, 32, 5.0, 0.15),
    ("hyper16_67x45_S6", lambda: synthetic.hyperspectral_mixture(67, 45, 16, seed=26), False, 16, 2.0, 0.2),
    ("rgb_40x33_S2", lambda: synthetic.color_rectangles(40, 33, seed=27), False, 5, 0.6, 0.1),
]


def _guide_for(f, separate):
    if not separate:
        return f
    g, _, _ = O.pca_guide(f.astype(np.float64), 7, 6)
    return g.astype(np.float32)


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("coef", ["opt", "indicator"])
def test_apply_matches_oracle(api, case, coef):
    name, make, separate, K, ss, sr = case
    f = make()
    p = _guide_for(f, separate)
    mu = _centres(p, K)
    S = O.window_halfwidth(ss)
    ref = O.fast_filter(f, p, mu.astype(np.float64), ss, sr, S, variant=coef)
    n, H, W = f.shape
    flt = api.HDFilter(H, W, n, p.shape[0], K, ss, sr, coef=coef)
    flt.set_centers(mu)
    fd = _cuda(f)
    pd = fd if not separate else _cuda(p)
    g = flt.apply(fd, pd).cpu().numpy()
    st = flt.stats()
    assert st["K_eff"] == mu.shape[0]
    err = np.max(np.abs(g - ref))
    assert err <= TOL, (name, err)


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_bruteforce_matches_oracle(api, case):
    name, make, separate, K, ss, sr = case
    f = make()
    p = _guide_for(f, separate)
    S = O.window_halfwidth(ss)
    ref = O.bruteforce(f, p, ss, sr, S)
    fd = _cuda(f)
    pd = fd if not separate else _cuda(p)
    g = api.bruteforce(fd, pd, ss, sr, S).cpu().numpy()
    assert np.max(np.abs(g - ref)) <= TOL


@pytest.mark.parametrize("dup", [False, True])
def test_pinv_matches_oracle(api, dup):
    rng = np.random.default_rng(31)
    mu = rng.uniform(size=(9, 3)).astype(np.float32)
    if dup:
        mu[6] = mu[2]
    flt = api.HDFilter(16, 16, 3, 3, 9, 1.0, 0.4)
    flt.set_centers(mu)
    got = flt.get_pinv()
    ref = O.pinv_psd(O.kernel_matrix(mu.astype(np.float64), 0.4))
    scale = np.abs(ref).max()
    assert np.max(np.abs(got - ref)) <= 1e-9 * scale


def test_rank_deficient_filter_matches_oracle(api):
    f = synthetic.color_rectangles(64, 48, seed=32)
    mu = _centres(f, 6)
    mu = np.concatenate([mu, mu[1:2]])            # duplicate centre: singular A
    ref = O.fast_filter(f, f, mu.astype(np.float64), 2.0, 0.2, 6)
    flt = api.HDFilter(64, 48, 3, 3, 7, 2.0, 0.2)
    flt.set_centers(mu)
    g = flt.apply(_cuda(f)).cpu().numpy()
    assert np.max(np.abs(g - ref)) <= TOL


@pytest.mark.parametrize("shape", [(3, 1, 1), (3, 1, 57), (1, 45, 1), (2, 5, 7), (3, 33, 64)])
def test_degenerate_shapes(api, shape):
    rng = np.random.default_rng(33)
    f = rng.uniform(size=shape).astype(np.float32)
    n, H, W = shape
    K = min(4, H * W)
    mu = _centres(f, K)
    ref = O.fast_filter(f, f, mu.astype(np.float64), 3.0, 0.3, 9)
    flt = api.HDFilter(H, W, n, n, K, 3.0, 0.3)
    flt.set_centers(mu)
    g = flt.apply(_cuda(f)).cpu().numpy()
    assert np.max(np.abs(g - ref)) <= TOL
    gb = api.bruteforce(_cuda(f), None, 3.0, 0.3).cpu().numpy()
    assert np.max(np.abs(gb - O.bruteforce(f, f, 3.0, 0.3, 9))) <= TOL


@pytest.mark.parametrize("S", [3, 9, 15, 24])
@pytest.mark.parametrize("spatial", ["gauss", "box"])
def test_word_and_vector_staging_agree(api, S, spatial):
    """The tile kernel stages its halo rows by 16-byte copies when W % 4 == 0
    and the image is 16-byte aligned, by single words otherwise: an image
    stored one float past an aligned address takes the word path, and the
    staged values and the arithmetic are the same, so the results are equal
    bit for bit; both match the oracle."""
    f = synthetic.color_rectangles(72, 96, seed=34)
    n, H, W = f.shape
    mu = _centres(f, 6)
    flt = api.HDFilter(H, W, n, n, 6, S / 3.0, 0.2, S=S, spatial=spatial)
    flt.set_centers(mu)
    fa = _cuda(f)
    buf = torch.empty(fa.numel() + 1, device="cuda", dtype=torch.float32)
    fm = buf[1:].view(n, H, W)
    fm.copy_(fa)
    assert fm.data_ptr() % 16 != 0 and fa.data_ptr() % 16 == 0
    ga = flt.apply(fa).cpu()
    gm = flt.apply(fm).cpu()
    assert torch.equal(ga, gm)
    ref = O.fast_filter(f, f, mu.astype(np.float64), S / 3.0, 0.2, S, spatial=spatial)
    assert float(np.max(np.abs(ga.numpy() - ref))) <= TOL


def test_constant_image_returned_unchanged(api):
    f = np.full((3, 70, 90), 0.4375, dtype=np.float32)
    flt = api.HDFilter(70, 90, 3, 3, 8, 3.0, 0.2)
    flt.set_centers(f[:, :1, 0].T.copy())
    g = flt.apply(_cuda(f)).cpu().numpy()
    assert np.max(np.abs(g - f)) <= 1e-6


def test_full_size_hyperspectral_sampled(api):
    w = synthetic.workload("hyper512")
    f = w["f"]
    mu = _centres(f, w["K"])
    S = O.window_halfwidth(w["sigma_s"])
    flt = api.HDFilter(512, 512, 31, 31, w["K"], w["sigma_s"], w["sigma_r"])
    flt.set_centers(mu)
    g = flt.apply(_cuda(f)).cpu().numpy()
    rng = np.random.default_rng(34)
    pix = np.concatenate([rng.integers(0, 512, size=(40, 2)),
                          np.array([[0, 0], [511, 511], [0, 511], [255, 256], [63, 64]])])
    ref = O.fast_filter_at(f, f, mu.astype(np.float64), w["sigma_s"], w["sigma_r"], S, pix)
    got = g[:, pix[:, 0], pix[:, 1]].T
    assert np.max(np.abs(got - ref)) <= TOL
    assert flt.stats()["fallback_pixels"] == 0
