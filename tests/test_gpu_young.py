"""GPU parity of the recursive-Gaussian mode (HDF_SPATIAL_YOUNG: Young and van
Vliet's O(1) recursion, the convolution Sec. II-C names) against the FP64
oracle's recursion, element by element, on ragged shapes; the calls that
do not support the mode refuse it.  The CUDA path gets the oracle's
centres; tolerance max-abs <= 1e-4 (the float recursion's error grows like
1/B, about 150 at sigma_s = 8; the cases stay at sigma_s <= 8)."""
import ctypes as C

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
    # name, image maker, K, sigma_s, sigma_r
    ("rgb_90x77_s2", lambda: synthetic.color_rectangles(90, 77, seed=101), 8, 2.0, 0.2),
    ("rgb_70x130_s5", lambda: synthetic.color_rectangles(70, 130, seed=102), 12, 5.0, 0.2),
    ("hyper16_64x50_s3", lambda: synthetic.hyperspectral_mixture(64, 50, 16, seed=103), 16, 3.0, 0.25),
    ("gray_100x96_s8", lambda: synthetic.smooth_field_with_edges(100, 96, seed=104), 8, 8.0, 0.15),
    ("rgb_33x40_s0.7", lambda: synthetic.color_rectangles(33, 40, seed=105), 6, 0.7, 0.2),
    ("hyper31_96x64_s5", lambda: synthetic.hyperspectral_mixture(96, 64, 31, seed=106), 32, 5.0, 0.3),
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
@pytest.mark.parametrize("coef", ["opt", "indicator"])
def test_young_apply_matches_oracle(api, case, coef):
    name, make, K, ss, sr = case
    f = make()
    mu = _centres(f, K)
    ref = O.fast_filter(f, f, mu.astype(np.float64), ss, sr, 0, variant=coef, spatial="young")
    n, H, W = f.shape
    flt = api.HDFilter(H, W, n, n, K, ss, sr, coef=coef, spatial="young")
    flt.set_centers(mu)
    g = flt.apply(_cuda(f)).cpu().numpy()
    assert flt.stats()["device_error"] == 0
    err = float(np.max(np.abs(g - ref)))
    assert err <= TOL, (name, err)


def test_young_separate_guide_and_clustering_on_device(api):
    f = synthetic.smooth_field_with_edges(80, 72, seed=107)
    p, _, _ = O.pca_guide(f.astype(np.float64), 5, 4)
    p = p.astype(np.float32)
    flt = api.HDFilter(80, 72, 1, 4, 16, 4.0, 0.15, spatial="young")
    pd = _cuda(p)
    flt.cluster(pd)
    mu = flt.get_centers()
    g = flt.apply(_cuda(f), pd).cpu().numpy()
    ref = O.fast_filter(f, p, mu.astype(np.float64), 4.0, 0.15, 0, spatial="young")
    assert float(np.max(np.abs(g - ref))) <= TOL


def test_young_is_refused_where_unsupported(api):
    from paper_1811_02363_gb300 import _lib as L
    d = api.make_desc(20, 24, 3, 3, 4, 0.4, 0.2, spatial="young")   # sigma_s < 0.5
    h = C.c_void_p()
    assert L.lib().hdf_create(C.byref(h), C.byref(d)) == L.HDF_EINVAL
    with pytest.raises(Exception):
        api.Batch([dict(H=20, W=24, n=3, K=4, sigma_s=2.0, sigma_r=0.2, spatial="young")])
    f = synthetic.color_rectangles(20, 24, seed=108)
    flt = api.HDFilter(20, 24, 3, 3, 4, 2.0, 0.2, spatial="young")
    flt.set_centers(_centres(f, 4))
    fd = _cuda(f)
    with pytest.raises(Exception):
        flt.backward(fd, fd, torch.ones_like(fd))
    mu = torch.from_numpy(_centres(f, 4)).cuda()
    g = torch.empty_like(fd)
    d2 = api.make_desc(20, 24, 3, 3, 4, 2.0, 0.2, spatial="young")
    st = L.lib().hdf_apply_static(C.byref(d2), C.c_void_p(mu.data_ptr()), 4, C.c_void_p(fd.data_ptr()),
                                  C.c_void_p(fd.data_ptr()), C.c_void_p(g.data_ptr()), None)
    assert st == L.HDF_EUNSUPPORTED
