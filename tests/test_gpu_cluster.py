"""GPU bisecting K-means (Sec. II-C) against the FP64 oracle.

Exact cases (distinct values, constant data) must match exactly; on noisy
data the centres must match within 1e-5 relative, the cluster error E_K
within 1e-6 relative, and at least 99.9 % of the labels must agree (the
coordinate sums behind the means are accumulated in a different order, so
points within rounding of a decision boundary may go the other way)."""
import numpy as np
import pytest
import torch

from oracle import hdfilter_oracle as O
from paper_1811_02363_gb300 import synthetic

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def api():
    from paper_1811_02363_gb300 import build
    build.build()
    from paper_1811_02363_gb300 import api as A
    return A


def _run(api, p, K, sigma_r=0.2, dtype=torch.float32):
    rho, H, W = p.shape
    flt = api.HDFilter(H, W, rho, rho, K, 1.0, sigma_r, guide_dtype="f32" if dtype == torch.float32 else "bf16")
    pd = torch.from_numpy(np.ascontiguousarray(p)).cuda().to(dtype)
    flt.cluster(pd)
    mu = flt.get_centers()
    lab = flt.get_labels().cpu().numpy()
    st = flt.stats()
    return flt, mu, lab, st


def _oracle(p, K):
    P = p.reshape(p.shape[0], -1).T.astype(np.float64)
    mu, lab, sse = O.bisecting_kmeans(P, K)
    return mu, lab, float(sse.sum()), P


def test_distinct_values_are_isolated_exactly(api):
    rng = np.random.default_rng(41)
    vals = rng.uniform(size=(7, 3)).astype(np.float32)
    lab = rng.integers(0, 7, size=(37, 29))
    lab.flat[:7] = np.arange(7)
    p = np.moveaxis(vals[lab], -1, 0).astype(np.float32)
    _, mu, glab, st = _run(api, p, 7)
    omu, olab, oek, _ = _oracle(p, 7)
    assert st["K_eff"] == 7 and st["device_error"] == 0
    assert np.array_equal(mu.astype(np.float64), omu)
    assert np.array_equal(glab, olab)
    assert st["cluster_error"] == 0.0


def test_constant_guide_single_cluster(api):
    p = np.full((3, 40, 50), 0.3, dtype=np.float32)
    _, mu, glab, st = _run(api, p, 8)
    assert st["K_eff"] == 1 and np.all(glab == 0)
    assert np.array_equal(mu, p[:, :1, 0].T)


def test_K_one(api):
    p = synthetic.color_rectangles(30, 20, seed=42)
    _, mu, glab, st = _run(api, p, 1)
    assert st["K_eff"] == 1 and np.all(glab == 0)
    assert np.allclose(mu[0], p.reshape(3, -1).mean(1), rtol=1e-5)


CASES = [
    ("rgb_96x80_K8", lambda: synthetic.color_rectangles(96, 80, seed=43), 8),
    ("rgb_150x97_K16", lambda: synthetic.color_rectangles(150, 97, seed=44), 16),
    ("hyper31_64x64_K32", lambda: synthetic.hyperspectral_mixture(64, 64, 31, seed=45), 32),
    ("hyper16_70x50_K16", lambda: synthetic.hyperspectral_mixture(70, 50, 16, seed=46), 16),
    ("gray_pca6_64x80_K32", lambda: O.pca_guide(synthetic.smooth_field_with_edges(64, 80, seed=47).astype(np.float64), 7, 6)[0].astype(np.float32), 32),
    ("rgb_200x300_K64", lambda: synthetic.color_rectangles(200, 300, seed=48), 64),
]


def _compare(mu, glab, st, omu, olab, oek):
    assert st["device_error"] == 0
    assert st["K_eff"] == omu.shape[0]
    agree = np.mean(glab == olab)
    assert agree >= 0.999, agree
    scale = np.abs(omu).max()
    assert np.max(np.abs(mu - omu)) <= 1e-5 * scale
    assert abs(st["cluster_error"] - oek) <= 1e-6 * oek


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_matches_oracle(api, case):
    name, make, K = case
    p = make()
    _, mu, glab, st = _run(api, p, K)
    omu, olab, oek, _ = _oracle(p, K)
    _compare(mu, glab, st, omu, olab, oek)


def test_repeatable(api):
    p = synthetic.hyperspectral_mixture(64, 64, 31, seed=49)
    flt, mu1, lab1, st1 = _run(api, p, 32)
    pd = torch.from_numpy(p).cuda()
    flt.cluster(pd)
    assert np.array_equal(flt.get_centers(), mu1)
    assert np.array_equal(flt.get_labels().cpu().numpy(), lab1)


def test_bf16_guide_matches_oracle_on_rounded_guide(api):
    p = synthetic.color_rectangles(120, 90, seed=50)
    pb = torch.from_numpy(p).to(torch.bfloat16)
    p_r = pb.to(torch.float32).numpy()
    _, mu, glab, st = _run(api, p_r, 12, dtype=torch.bfloat16)
    omu, olab, oek, _ = _oracle(p_r, 12)
    _compare(mu, glab, st, omu, olab, oek)


def test_full_size_hyperspectral(api):
    w = synthetic.workload("hyper512")
    p = w["f"]
    _, mu, glab, st = _run(api, p, w["K"], w["sigma_r"])
    omu, olab, oek, _ = _oracle(p, w["K"])
    _compare(mu, glab, st, omu, olab, oek)
