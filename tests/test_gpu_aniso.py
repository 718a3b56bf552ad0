"""The anisotropic range kernel on the device (Sec. III-E): the guide scaled
per dimension by hdf_scale_guide and sigma_r = 1 against the FP64 oracle's
anisotropic kernel exp(-sum_d x_d^2 / (2 sigma_{r,d}^2)) on the unscaled
guide, for Algorithm 1 and for the brute force; then the low-light + infrared
nonlocal-means case of Sec. III-E (7x7 patches of the dark frame reduced to
6 PCA features on the device, the infrared frame as a seventh dimension,
sigma_r 50/255 for the first six and 10/255 for the infrared one, a 17x17
box search window, K = 32).  Tolerance: max-abs <= 1e-4."""
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
    return A


def test_scale_guide_divides_each_dimension(api):
    f = synthetic.color_rectangles(33, 47, seed=51)
    sr = [0.1, 0.25, 0.4]
    q = api.scale_guide(torch.from_numpy(f).cuda(), sr).cpu().numpy()
    assert np.max(np.abs(q - O.scaled_guide(f, sr))) <= 1e-6 * np.abs(q).max()


@pytest.mark.parametrize("coef", ["opt", "indicator"])
def test_anisotropic_filter_matches_oracle(api, coef):
    f = synthetic.color_rectangles(96, 80, seed=52)
    n, H, W = f.shape
    sr = np.array([0.1, 0.3, 0.2])
    fd = torch.from_numpy(f).cuda()
    q = api.scale_guide(fd, sr)
    qn = O.scaled_guide(f, sr)
    mu_s = O.bisecting_kmeans(qn.reshape(n, -1).T, 10)[0].astype(np.float32)   # scaled units
    flt = api.HDFilter(H, W, n, n, 10, 3.0, 1.0, coef=coef)
    flt.set_centers(mu_s)
    g = flt.apply(fd, q).cpu().numpy()
    mu = mu_s.astype(np.float64) * sr[None, :]                               # original units
    ref = O.fast_filter(f, f, mu, 3.0, sr, 9, variant=coef)
    assert float(np.max(np.abs(g - ref))) <= TOL
    gb = api.bruteforce(fd, q, 3.0, 1.0).cpu().numpy()
    assert float(np.max(np.abs(gb - O.bruteforce(f, f, 3.0, sr, 9)))) <= TOL


def test_lowlight_with_infrared_guide(api):
    H = W = 256
    dark, ir = synthetic.lowlight_infrared(H, W, seed=53)
    sr = np.array([50.0 / 255] * 6 + [10.0 / 255])
    fd = torch.from_numpy(dark).cuda()
    flt = api.HDFilter(H, W, 1, 7, 32, 8.0 / 3.0, 1.0, S=8, spatial="box")
    p = torch.empty((7, H, W), device="cuda")
    guide6 = api.HDFilter(H, W, 1, 6, 32, 8.0 / 3.0, 1.0, S=8, spatial="box")
    guide6.nlm_guide(fd, 7, out=p[:6])
    p[6].copy_(torch.from_numpy(ir[0]).cuda())
    q = api.scale_guide(p, sr)
    flt.cluster(q)
    g = flt.apply(fd, q).cpu().numpy()
    st = flt.stats()
    assert st["device_error"] == 0 and st["K_eff"] == 32
    mu = flt.get_centers().astype(np.float64) * sr[None, :]
    pn = p.cpu().numpy().astype(np.float64)
    ref = O.fast_filter(dark, pn, mu, 8.0 / 3.0, sr, 8, spatial="box")
    assert float(np.max(np.abs(g - ref))) <= TOL
    # the infrared dimension sharpens the result: closer to the scene than the
    # same filter with the low-light features alone (a qualitative check)
    guide6.close()
    flt.close()
