"""GPU parity of the batch path -- many images of different sizes, channel
counts, window sizes and centre counts through one launch per stage, the
persistent tile launch, CUDA-graph replay and tuned tile shapes -- against
the FP64 oracle, image by image.

As in the single-image tests the filter is compared with the oracle given
the oracle's own centres (installed with set_centers); the batch clustering
is compared with the oracle's bisecting K-means on the same guide.
Tolerance for the float32 paths: max-abs <= 1e-4."""
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


def _bf16_round(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(torch.bfloat16).to(torch.float32).numpy()


# (maker, sigma_s, sigma_r, K): every window bucket, 1 / 3 / 16 channels,
# sides that are not multiples of the tile, one image smaller than a tile.
MIX = [
    (lambda: synthetic.color_rectangles(70, 45, seed=61), 1.3, 0.2, 8),
    (lambda: synthetic.hyperspectral_mixture(37, 90, 16, seed=62), 2.5, 0.25, 16),
    (lambda: synthetic.smooth_field_with_edges(64, 64, seed=63), 4.0, 0.15, 4),
    (lambda: synthetic.color_rectangles(33, 129, seed=64), 5.0, 0.3, 12),
    (lambda: synthetic.color_rectangles(100, 41, seed=65), 6.0, 0.2, 8),
    (lambda: synthetic.hyperspectral_mixture(50, 50, 16, seed=66), 7.5, 0.2, 32),
    (lambda: synthetic.color_rectangles(20, 90, seed=67), 10.5, 0.25, 6),
    (lambda: synthetic.color_rectangles(9, 7, seed=68), 0.9, 0.2, 5),
]


def _images(mix):
    out = []
    for make, ss, sr, K in mix:
        f = np.ascontiguousarray(make(), dtype=np.float32)
        out.append((f, ss, sr, K))
    return out


def _specs(images, guide_dtype="f32"):
    return [dict(H=f.shape[1], W=f.shape[2], n=f.shape[0], K=K, sigma_s=ss, sigma_r=sr,
                 guide_dtype=guide_dtype) for f, ss, sr, K in images]


def _oracle_outputs(images, mus, guides=None):
    refs = []
    for i, (f, ss, sr, K) in enumerate(images):
        p = f if guides is None else guides[i]
        refs.append(O.fast_filter(f, p, mus[i].astype(np.float64), ss, sr,
                                  O.window_halfwidth(ss)))
    return refs


@pytest.fixture(scope="module")
def mixed(api):
    images = _images(MIX)
    mus = [_centres(f, K) for f, _, _, K in images]
    refs = _oracle_outputs(images, mus)
    return images, mus, refs


def _bound_batch(api, images, mus=None, guide_dtype="f32"):
    b = api.Batch(_specs(images, guide_dtype))
    fs = [_cuda(f) for f, *_ in images]
    gs = [torch.empty_like(f) for f in fs]
    b.bind(fs, gs)
    if mus is not None:
        for i, mu in enumerate(mus):
            b.set_centers(i, mu)
    return b, fs, gs


def _check(gs, refs, images, b=None):
    for i, (g, ref) in enumerate(zip(gs, refs)):
        err = float(np.max(np.abs(g.cpu().numpy() - ref)))
        assert err <= TOL, (i, images[i][0].shape, err)
        if b is not None:
            assert b.stats(i)["device_error"] == 0


def test_mixed_batch_matches_oracle_eager_and_graph(api, mixed):
    images, mus, refs = mixed
    b, fs, gs = _bound_batch(api, images, mus)
    b.run(graph=False)
    torch.cuda.synchronize()
    _check(gs, refs, images, b)
    eager = [g.clone() for g in gs]
    for g in gs:
        g.fill_(-1.0)
    b.run(graph=True)
    b.run(graph=True)   # replay
    torch.cuda.synchronize()
    info = b.info()
    assert info["graph_state"] == 1, info
    for g, e in zip(gs, eager):
        assert torch.equal(g, e)
    assert info["nitems"] > 0 and info["grid_tile"] >= torch.cuda.get_device_properties(0).multi_processor_count


def test_every_compiled_tile_shape_matches_oracle(api, mixed):
    images, mus, refs = mixed
    b, fs, gs = _bound_batch(api, images, mus)
    trials = b.tune(reps=1)
    keys = {(t["SB"], t["planes"]) for t in trials}
    assert len(keys) == len({(t["SB"], t["planes"]) for t in trials if t["chosen"]})
    for key in keys:
        assert sum(t["chosen"] for t in trials if (t["SB"], t["planes"]) == key) == 1
    assert all(t["ms"] > 0 for t in trials)
    b.run(graph=False)
    torch.cuda.synchronize()
    _check(gs, refs, images, b)   # tuned shapes
    for t in trials:
        b.set_shape(t["SB"], t["planes"], t["P"], t["TY"])
        for g in gs:
            g.fill_(-1.0)
        b.run(graph=False)
        torch.cuda.synchronize()
        _check(gs, refs, images)


def test_timed_run_reports_stages(api, mixed):
    images, mus, refs = mixed
    b, fs, gs = _bound_batch(api, images, mus)
    b.run(graph=False, timed=True)
    t = b.times()
    assert len(t) == 7 and all(x >= 0 for x in t)
    assert t[5] > 0   # the persistent tile launch
    _check(gs, refs, images, b)


def test_batch_clustering_matches_oracle(api):
    images = _images([
        (lambda: synthetic.color_rectangles(96, 80, seed=71), 3.0, 0.2, 8),
        (lambda: synthetic.hyperspectral_mixture(64, 64, 16, seed=72), 2.0, 0.2, 16),
        (lambda: synthetic.color_rectangles(150, 97, seed=73), 5.0, 0.25, 32),
        (lambda: synthetic.hyperspectral_mixture(70, 50, 16, seed=74), 6.0, 0.3, 8),
        (lambda: np.full((3, 30, 40), 0.3, np.float32), 2.0, 0.2, 8),
    ])
    b, fs, gs = _bound_batch(api, images)
    b.run(graph=True)
    torch.cuda.synchronize()
    for i, (f, ss, sr, K) in enumerate(images):
        omu, _, sse = O.bisecting_kmeans(f.reshape(f.shape[0], -1).T.astype(np.float64), K)
        st = b.stats(i)
        mu = b.get_centers(i)
        assert st["device_error"] == 0 and st["K_eff"] == omu.shape[0], (i, st)
        scale = max(np.abs(omu).max(), 1e-30)
        assert np.max(np.abs(mu - omu)) <= 1e-5 * scale, i
        oek = float(sse.sum())
        assert abs(st["cluster_error"] - oek) <= 1e-6 * oek, (i, st["cluster_error"], oek)


def test_tuned_clustering_plan_matches_oracle(api):
    """The tuner times the clustering launch under every plan (a group per
    image, or M equal groups taking their images in turn), keeps one, and the
    batch run under the kept plan still matches the oracle's clustering."""
    images = _images([
        (lambda: synthetic.color_rectangles(96, 80, seed=81), 3.0, 0.2, 8),
        (lambda: synthetic.hyperspectral_mixture(64, 64, 16, seed=82), 2.0, 0.2, 16),
        (lambda: synthetic.color_rectangles(150, 97, seed=83), 5.0, 0.25, 32),
        (lambda: synthetic.hyperspectral_mixture(70, 50, 16, seed=84), 6.0, 0.3, 8),
        (lambda: synthetic.color_rectangles(40, 33, seed=85), 2.0, 0.2, 4),
    ])
    b, fs, gs = _bound_batch(api, images)
    trials = [t for t in b.tune(reps=1) if t["SB"] == 0]
    assert [t["planes"] for t in trials] == [0, 1, 2, 4]
    assert sum(t["chosen"] for t in trials) == 1 and all(t["ms"] > 0 for t in trials)
    b.run(graph=True)
    torch.cuda.synchronize()
    for i, (f, ss, sr, K) in enumerate(images):
        omu, _, sse = O.bisecting_kmeans(f.reshape(f.shape[0], -1).T.astype(np.float64), K)
        st = b.stats(i)
        mu = b.get_centers(i)
        assert st["device_error"] == 0 and st["K_eff"] == omu.shape[0], (i, st)
        assert np.max(np.abs(mu - omu)) <= 1e-5 * max(np.abs(omu).max(), 1e-30), i
        oek = float(sse.sum())
        assert abs(st["cluster_error"] - oek) <= 1e-6 * oek, (i, st["cluster_error"], oek)


def test_more_images_than_sms(api):
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    count = sms + 9
    rng = np.random.default_rng(75)
    images = []
    for i in range(count):
        H, W = int(rng.integers(6, 20)), int(rng.integers(6, 20))
        images.append((synthetic.color_rectangles(H, W, n_rect=3, seed=1000 + i), 1.0, 0.2, 4))
    b, fs, gs = _bound_batch(api, images)
    b.run(graph=True)
    torch.cuda.synchronize()
    info = b.info()
    # more images than 8: four equal block groups, each taking its images in turn
    assert info["ngroups"] == 4 and info["grid_cluster"] == 4 * (sms // 4)
    mus = [_centres(f, K) for f, _, _, K in images]
    for i in range(count):
        mu = b.get_centers(i)
        assert mu.shape == mus[i].shape, i
        assert np.max(np.abs(mu - mus[i])) <= 1e-5 * np.abs(mus[i]).max(), i
    # the filter of every image with the oracle's centres
    b2, fs2, gs2 = _bound_batch(api, images, mus)
    b2.run(graph=True)
    torch.cuda.synchronize()
    _check(gs2, _oracle_outputs(images, mus), images)


def test_bf16_guide_storage_matches_oracle_on_rounded_guide(api):
    images = _images([
        (lambda: synthetic.color_rectangles(80, 60, seed=81), 2.0, 0.2, 8),
        (lambda: synthetic.hyperspectral_mixture(45, 70, 16, seed=82), 3.0, 0.25, 16),
        (lambda: synthetic.color_rectangles(33, 65, seed=83), 5.0, 0.15, 12),
    ])
    guides = [_bf16_round(f) for f, *_ in images]
    mus = [_centres(p, K) for p, (_, _, _, K) in zip(guides, images)]
    refs = _oracle_outputs(images, mus, guides)
    b, fs, gs = _bound_batch(api, images, mus, guide_dtype="bf16")
    b.run(graph=True)
    torch.cuda.synchronize()
    _check(gs, refs, images, b)
    # clustering from the bfloat16 guide the run stores
    b2, fs2, gs2 = _bound_batch(api, images, None, guide_dtype="bf16")
    b2.run(graph=True)
    torch.cuda.synchronize()
    for i, (p, (_, _, _, K)) in enumerate(zip(guides, images)):
        omu, _, _ = O.bisecting_kmeans(p.reshape(p.shape[0], -1).T.astype(np.float64), K)
        mu = b2.get_centers(i)
        assert np.max(np.abs(mu - omu)) <= 1e-5 * np.abs(omu).max(), i


def test_single_image_bf16_guide_filter_matches_oracle(api):
    f = synthetic.color_rectangles(90, 70, seed=84)
    p = _bf16_round(f)
    mu = _centres(p, 10)
    ref = O.fast_filter(f, p, mu.astype(np.float64), 3.0, 0.2, 9)
    flt = api.HDFilter(90, 70, 3, 3, 10, 3.0, 0.2, guide_dtype="bf16")
    flt.set_centers(mu)
    g = flt.apply(_cuda(f), _cuda(f, torch.bfloat16)).cpu().numpy()
    assert np.max(np.abs(g - ref)) <= TOL


def test_serving_batch_full_size_sampled(api):
    """The 64-image serving workload at full size (sides 256..2048, RGB and
    16-band, sigma_s in [2, 8], K in {8, 16, 32}, bfloat16 guide storage), in
    the launch configuration the benchmark times: clustering on the device
    for every image, then the filter with centres the oracle computes on a
    pixel subsample, checked at sampled pixels."""
    items = synthetic.serving_batch(64, seed=4)
    images = [(it.image, it.sigma_s, it.sigma_r, it.K) for it in items]
    b, fs, gs = _bound_batch(api, images, None, guide_dtype="bf16")
    b.run(graph=True)
    torch.cuda.synchronize()
    for i, (f, ss, sr, K) in enumerate(images):
        st = b.stats(i)
        assert st["device_error"] == 0 and st["K_eff"] == K, (i, st)
    rng = np.random.default_rng(85)
    mus, guides = [], []
    for f, ss, sr, K in images:
        n, H, W = f.shape
        p = _bf16_round(f)
        sub = rng.choice(H * W, size=min(H * W, 4096), replace=False)
        P = p.reshape(n, -1)[:, sub].T.astype(np.float64)
        mu, _, _ = O.bisecting_kmeans(P, K)
        mus.append(mu.astype(np.float32))
        guides.append(p)
    for i, mu in enumerate(mus):
        b.set_centers(i, mu)
    b.run(graph=True)
    torch.cuda.synchronize()
    for i, (f, ss, sr, K) in enumerate(images):
        n, H, W = f.shape
        pix = np.concatenate([rng.integers(0, [H, W], size=(4, 2)),
                              np.array([[0, 0], [H - 1, W - 1]])])
        ref = O.fast_filter_at(f, guides[i], mus[i].astype(np.float64), ss, sr,
                               O.window_halfwidth(ss), pix)
        got = gs[i][:, pix[:, 0], pix[:, 1]].T.cpu().numpy()
        assert np.max(np.abs(got - ref)) <= TOL, i
