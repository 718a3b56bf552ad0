"""GPU parity of the box spatial kernel (omega = 1 on W = [-S, S]^2, the kernel
Sec. III uses for nonlocal means) against the FP64 oracle: the fast filter
(running-sum convolutions in the tile kernel), the brute force, the guard,
the batch path, and the full-size nonlocal-means workload with the paper's
box half-width S = 10 checked at sampled pixels.  The CUDA path gets the
oracle's centres; tolerance max-abs <= 1e-4 (float32 paths)."""
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


def _cuda(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=torch.float32)


def _centres(p, K):
    mu, _, _ = O.bisecting_kmeans(p.reshape(p.shape[0], -1).T.astype(np.float64), K)
    return mu.astype(np.float32)


CASES = [
    # name, image maker, K, S (the box half-width), sigma_r
    ("rgb_90x77_S2", lambda: synthetic.color_rectangles(90, 77, seed=91), 8, 2, 0.2),
    ("rgb_70x130_S10", lambda: synthetic.color_rectangles(70, 130, seed=92), 12, 10, 0.2),
    ("hyper16_64x50_S7", lambda: synthetic.hyperspectral_mixture(64, 50, 16, seed=93), 16, 7, 0.25),
    ("gray_100x96_S15", lambda: synthetic.smooth_field_with_edges(100, 96, seed=94), 8, 15, 0.15),
    ("rgb_33x40_S24", lambda: synthetic.color_rectangles(33, 40, seed=95), 6, 24, 0.2),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("coef", ["opt", "indicator"])
def test_box_apply_matches_oracle(api, case, coef):
    name, make, K, S, sr = case
    f = make()
    mu = _centres(f, K)
    ref = O.fast_filter(f, f, mu.astype(np.float64), 1.0, sr, S, variant=coef, spatial="box")
    n, H, W = f.shape
    flt = api.HDFilter(H, W, n, n, K, 1.0, sr, S=S, coef=coef, spatial="box")
    flt.set_centers(mu)
    g = flt.apply(_cuda(f)).cpu().numpy()
    assert flt.stats()["device_error"] == 0
    err = float(np.max(np.abs(g - ref)))
    assert err <= TOL, (name, err)


@pytest.mark.parametrize("case", CASES[:3], ids=[c[0] for c in CASES[:3]])
def test_box_bruteforce_matches_oracle(api, case):
    name, make, K, S, sr = case
    f = make()
    ref = O.bruteforce(f, f, 1.0, sr, S, spatial="box")
    g = api.bruteforce(_cuda(f), None, 1.0, sr, S=S, spatial="box").cpu().numpy()
    assert float(np.max(np.abs(g - ref))) <= TOL, name


def test_box_fast_equals_box_bruteforce_with_a_centre_per_value(api):
    rng = np.random.default_rng(96)
    vals = rng.uniform(size=(6, 3)).astype(np.float32)
    lab = rng.integers(0, 6, size=(40, 50))
    lab.flat[:6] = np.arange(6)
    f = np.ascontiguousarray(np.moveaxis(vals[lab], -1, 0))
    flt = api.HDFilter(40, 50, 3, 3, 6, 1.0, 0.2, S=5, spatial="box")
    fd = _cuda(f)
    flt.cluster(fd)
    g = flt.apply(fd).cpu().numpy()
    gb = api.bruteforce(fd, None, 1.0, 0.2, S=5, spatial="box").cpu().numpy()
    assert flt.stats()["K_eff"] == 6
    assert float(np.max(np.abs(g - gb))) <= TOL


def test_box_backward_is_unsupported(api):
    f = synthetic.color_rectangles(20, 24, seed=97)
    flt = api.HDFilter(20, 24, 3, 3, 4, 1.0, 0.2, S=3, spatial="box")
    flt.set_centers(_centres(f, 4))
    fd = _cuda(f)
    with pytest.raises(Exception):
        flt.backward(fd, fd, torch.ones_like(fd))


def test_box_batch_matches_oracle(api):
    imgs = [(synthetic.color_rectangles(60, 70, seed=98), 6, 4, 0.2),
            (synthetic.hyperspectral_mixture(50, 44, 16, seed=99), 8, 9, 0.25)]
    specs, fs, gs, mus, refs = [], [], [], [], []
    for f, K, S, sr in imgs:
        n, H, W = f.shape
        specs.append(dict(H=H, W=W, n=n, K=K, sigma_s=1.0, sigma_r=sr, S=S, spatial="box"))
        mu = _centres(f, K)
        mus.append(mu)
        refs.append(O.fast_filter(f, f, mu.astype(np.float64), 1.0, sr, S, spatial="box"))
        fs.append(_cuda(f))
        gs.append(torch.empty_like(fs[-1]))
    b = api.Batch(specs)
    b.bind(fs, gs)
    for i, mu in enumerate(mus):
        b.set_centers(i, mu)
    b.run(graph=True)
    torch.cuda.synchronize()
    for g, ref in zip(gs, refs):
        assert float(np.max(np.abs(g.cpu().numpy() - ref))) <= TOL


def test_box_full_size_nlm_sampled(api):
    """The 1024 x 1024 nonlocal-means workload (guide: 7 x 7 patches reduced to
    6 PCA features on the device) with the paper's box window S = 10, K = 32,
    checked against the window-sum definition at sampled pixels."""
    w = synthetic.workload("nlm1024")
    f = w["f"]
    n, H, W = f.shape
    flt = api.HDFilter(H, W, n, 6, 32, 1.0, w["sigma_r"], S=10, spatial="box")
    fd = _cuda(f)
    p = flt.nlm_guide(fd, 7)
    flt.cluster(p)
    mu = flt.get_centers()
    g = flt.apply(fd, p).cpu().numpy()
    rng = np.random.default_rng(100)
    pix = np.stack([rng.integers(0, H, 48), rng.integers(0, W, 48)], axis=1)
    pix[:4] = [[0, 0], [H - 1, W - 1], [0, W - 1], [H - 1, 0]]
    ref = O.fast_filter_at(f, p.cpu().numpy(), mu.astype(np.float64), 1.0, w["sigma_r"], 10, pix,
                           spatial="box")
    got = g[:, pix[:, 0], pix[:, 1]].T
    assert float(np.max(np.abs(got - ref))) <= TOL
