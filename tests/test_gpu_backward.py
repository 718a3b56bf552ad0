"""GPU backward pass (dL/df, dL/dlog sigma_s, dL/dlog sigma_r with the centres
and S fixed) against the FP64 autograd reference of oracle/hdfilter_grad.py,
which is itself pinned by central differences.  Float32 tolerance: the
gradients are sums of O(K (2S+1)^2) float32 products, so they are compared
at 1e-3 of their largest magnitude (elementwise) and 1e-3 relative (scalars)."""
import math

import numpy as np
import pytest
import torch

from oracle import hdfilter_grad as OG
from oracle import hdfilter_oracle as O
from paper_1811_02363_gb300 import synthetic

pytestmark = pytest.mark.gpu
RTOL = 1e-3


@pytest.fixture(scope="module")
def api():
    from paper_1811_02363_gb300 import build
    build.build()
    from paper_1811_02363_gb300 import api as A
    return A


def _check(api, f, p, K, ss, sr, seed):
    rng = np.random.default_rng(seed)
    guide = f if p is None else p
    mu = O.bisecting_kmeans(guide.reshape(guide.shape[0], -1).T.astype(np.float64), K)[0].astype(np.float32)
    G = rng.normal(size=f.shape).astype(np.float32)
    S = O.window_halfwidth(ss)
    gf_ref, gls_ref, glr_ref, g_ref = OG.grads(f.astype(np.float64), None if p is None else p.astype(np.float64),
                                               mu.astype(np.float64), ss, sr, S, G.astype(np.float64))
    n, H, W = f.shape
    flt = api.HDFilter(H, W, n, guide.shape[0], mu.shape[0], ss, sr)
    flt.set_centers(mu)
    fd = torch.from_numpy(f).cuda()
    pd = fd if p is None else torch.from_numpy(p).cuda()
    gf, gls, glr = flt.backward(fd, pd, torch.from_numpy(G).cuda())
    st = flt.stats()
    assert st["fallback_pixels"] == 0 and st["device_error"] == 0
    gf = gf.cpu().numpy()
    scale = np.abs(gf_ref).max()
    assert np.max(np.abs(gf - gf_ref)) <= RTOL * scale, np.max(np.abs(gf - gf_ref)) / scale
    assert abs(float(gls) - gls_ref) <= RTOL * max(abs(gls_ref), 1e-3 * scale), (float(gls), gls_ref)
    assert abs(float(glr) - glr_ref) <= RTOL * max(abs(glr_ref), 1e-3 * scale), (float(glr), glr_ref)
    return flt


@pytest.mark.parametrize("shape,K,ss,sr", [((3, 40, 36), 5, 1.3, 0.35), ((3, 70, 45), 8, 2.0, 0.3),
                                          ((5, 33, 29), 6, 1.0, 0.4)])
def test_backward_guide_is_image(api, shape, K, ss, sr):
    n, H, W = shape
    if n == 3:
        f = synthetic.color_rectangles(H, W, seed=81)
    else:
        f = synthetic.hyperspectral_mixture(H, W, bands=n, seed=82)
    f = np.clip(f + np.random.default_rng(83).normal(0, 0.03, f.shape), 0, 1).astype(np.float32)
    _check(api, f, None, K, ss, sr, 84)


def test_backward_separate_guide(api):
    f = synthetic.color_rectangles(48, 40, seed=85)
    p = np.random.default_rng(86).uniform(size=(2, 48, 40)).astype(np.float32)
    _check(api, f, p, 6, 1.5, 0.3, 87)


def test_backward_crop_of_large_workload(api):
    # 64 x 64 crop of the 2048 x 2048 colour workload: K = 16, sigma_s = 8 (S = 24), sigma_r = 0.15
    f = synthetic.color_rectangles(2048, 2048, seed=3)[:, 700:764, 900:964].copy()
    f = np.clip(f + np.random.default_rng(88).normal(0, 0.02, f.shape), 0, 1).astype(np.float32)
    _check(api, f, None, 16, 8.0, 0.15, 89)


def test_autograd_function(api):
    f = synthetic.color_rectangles(40, 36, seed=90)
    mu = O.bisecting_kmeans(f.reshape(3, -1).T.astype(np.float64), 5)[0].astype(np.float32)
    flt = api.HDFilter(40, 36, 3, 3, 5, 1.3, 0.35)
    flt.set_centers(mu)
    fd = torch.from_numpy(f).cuda().requires_grad_(True)
    ls = torch.tensor(math.log(1.3), device="cuda", requires_grad=True)
    lr = torch.tensor(math.log(0.35), device="cuda", requires_grad=True)
    g = api.fast_filter(fd, ls, lr, flt)
    G = torch.from_numpy(np.random.default_rng(91).normal(size=f.shape).astype(np.float32)).cuda()
    (g * G).sum().backward()
    gf2, gls2, glr2 = flt.backward(fd.detach(), fd.detach(), G)
    assert torch.equal(fd.grad, gf2)
    assert float(ls.grad) == pytest.approx(float(gls2), rel=1e-6)
    assert float(lr.grad) == pytest.approx(float(glr2), rel=1e-6)


@pytest.mark.parametrize("ss", [1.3, 5.0, 8.0])
def test_backward_word_and_vector_staging_agree(api, ss):
    """The backward tile kernels stage halo rows by 16-byte copies when
    W % 4 == 0 and the image is 16-byte aligned, by single words otherwise;
    an image stored one float past an aligned address takes the word path and
    must give the same gradients bit for bit."""
    f = synthetic.color_rectangles(44, 48, seed=92)
    mu = O.bisecting_kmeans(f.reshape(3, -1).T.astype(np.float64), 6)[0].astype(np.float32)
    flt = api.HDFilter(44, 48, 3, 3, 6, ss, 0.3)
    flt.set_centers(mu)
    fa = torch.from_numpy(f).cuda()
    buf = torch.empty(fa.numel() + 1, device="cuda", dtype=torch.float32)
    fm = buf[1:].view(3, 44, 48)
    fm.copy_(fa)
    assert fm.data_ptr() % 16 != 0 and fa.data_ptr() % 16 == 0
    G = torch.from_numpy(np.random.default_rng(93).normal(size=f.shape).astype(np.float32)).cuda()
    ga, sa, ra = flt.backward(fa, fa, G)
    gm, sm, rm = flt.backward(fm, fm, G)
    assert torch.equal(ga, gm)
    assert float(sa) == float(sm) and float(ra) == float(rm)


def test_backward_equals_brute_force_gradients_at_exactness(api):
    """With a separate guide of 4 distinct values and one centre per value,
    Algorithm 1 equals the brute force for every f, sigma_s and sigma_r, so
    the device's backward pass must give the gradients of the brute force
    (FP64 autograd through Eq. (1)-(2))."""
    rng = np.random.default_rng(86)
    vals = rng.uniform(0, 1, size=(4, 2)).astype(np.float32)
    p = np.ascontiguousarray(np.moveaxis(vals[rng.integers(0, 4, size=(40, 37))], -1, 0))
    f = rng.uniform(0, 1, size=(3, 40, 37)).astype(np.float32)
    G = rng.normal(size=f.shape).astype(np.float32)
    ss, sr = 1.5, 0.3
    S = O.window_halfwidth(ss)
    bf, bls, blr, _ = OG.brute_grads(f.astype(np.float64), p.astype(np.float64), ss, sr, S,
                                     G.astype(np.float64))
    flt = api.HDFilter(40, 37, 3, 2, 4, ss, sr)
    flt.set_centers(vals)
    gf, gls, glr = flt.backward(torch.from_numpy(f).cuda(), torch.from_numpy(p).cuda(),
                                torch.from_numpy(G).cuda())
    gf = gf.cpu().numpy()
    scale = np.abs(bf).max()
    assert np.max(np.abs(gf - bf)) <= RTOL * scale
    assert abs(float(gls) - bls) <= RTOL * max(abs(bls), 1e-3 * scale)
    assert abs(float(glr) - blr) <= RTOL * max(abs(blr), 1e-3 * scale)


def test_set_sigmas_equals_a_handle_made_for_the_widths(api):
    """hdf_set_sigmas on a clustered handle (S and the centres kept, A^+
    refitted) gives bit for bit the filter of a handle created with the new
    widths, the same S and the same centres, and Algorithm 1 of the oracle at
    the new widths."""
    f = synthetic.color_rectangles(72, 61, seed=92)
    f = np.clip(f + np.random.default_rng(93).normal(0, 0.03, f.shape), 0, 1).astype(np.float32)
    fd = torch.from_numpy(f).cuda()
    S = 6
    flt = api.HDFilter(72, 61, 3, 3, 8, 2.0, 0.2, S=S)
    flt.cluster(fd)
    mu = flt.get_centers()
    flt.set_sigmas(2.6, 0.12)
    assert (flt.desc.sigma_s, flt.desc.sigma_r, flt.S) == (2.6, 0.12, S)
    g1 = flt.apply(fd, fd)
    ref = api.HDFilter(72, 61, 3, 3, mu.shape[0], 2.6, 0.12, S=S)
    ref.set_centers(mu)
    g2 = ref.apply(fd, fd)
    assert torch.equal(g1, g2)
    assert np.array_equal(flt.get_pinv(), ref.get_pinv())
    want = O.fast_filter(f.astype(np.float64), f.astype(np.float64), mu.astype(np.float64), 2.6, 0.12, S)
    assert np.max(np.abs(g1.cpu().numpy() - want)) <= 1e-4
    with pytest.raises(Exception):
        flt.set_sigmas(float("nan"), 0.1)
    with pytest.raises(Exception):
        flt.set_sigmas(1.0, 0.0)


def test_autograd_with_live_sigmas(api):
    """fast_filter installs the widths of its log-sigma inputs: the gradients
    at widths other than the handle's match the FP64 reference at those
    widths (S fixed), and a small step of log sigma_r against its gradient
    lowers the loss."""
    f = synthetic.color_rectangles(40, 36, seed=94)
    f = np.clip(f + np.random.default_rng(95).normal(0, 0.03, f.shape), 0, 1).astype(np.float32)
    mu = O.bisecting_kmeans(f.reshape(3, -1).T.astype(np.float64), 5)[0].astype(np.float32)
    flt = api.HDFilter(40, 36, 3, 3, 5, 1.3, 0.35)
    S = flt.S
    flt.set_centers(mu)
    G = np.random.default_rng(96).normal(size=f.shape).astype(np.float32)
    fd = torch.from_numpy(f).cuda().requires_grad_(True)
    ss, sr = 1.1, 0.28
    ls = torch.tensor(math.log(ss), device="cuda", dtype=torch.float64, requires_grad=True)
    lr = torch.tensor(math.log(sr), device="cuda", dtype=torch.float64, requires_grad=True)
    g = api.fast_filter(fd, ls, lr, flt)
    (g * torch.from_numpy(G).cuda()).sum().backward()
    gf_ref, gls_ref, glr_ref, g_ref = OG.grads(f.astype(np.float64), None, mu.astype(np.float64),
                                               ss, sr, S, G.astype(np.float64))
    assert np.max(np.abs(g.detach().cpu().numpy() - g_ref)) <= 1e-4
    scale = np.abs(gf_ref).max()
    assert np.max(np.abs(fd.grad.cpu().numpy() - gf_ref)) <= RTOL * scale
    assert abs(float(ls.grad) - gls_ref) <= RTOL * max(abs(gls_ref), 1e-3 * scale)
    assert abs(float(lr.grad) - glr_ref) <= RTOL * max(abs(glr_ref), 1e-3 * scale)
    assert ls.grad.dtype == torch.float64

    # descent on log sigma_r towards the output at sigma_r = 0.2
    target = O.fast_filter(f.astype(np.float64), f.astype(np.float64), mu.astype(np.float64),
                           1.3, 0.2, S)
    tgt = torch.from_numpy(target.astype(np.float32)).cuda()
    fx = torch.from_numpy(f).cuda()
    ls0 = torch.tensor(math.log(1.3), device="cuda")

    def loss_and_grad(v):
        lr_t = torch.tensor(v, device="cuda", requires_grad=True)
        L = ((api.fast_filter(fx, ls0, lr_t, flt) - tgt) ** 2).sum()
        L.backward()
        return float(L), float(lr_t.grad)

    v = math.log(0.35)
    L0, d0 = loss_and_grad(v)
    assert d0 > 0                                   # the loss grows with sigma_r above 0.2
    L1, _ = loss_and_grad(v - 0.1 * math.copysign(1.0, d0))
    assert L1 < L0


def test_backward_after_apply_equals_the_recomputing_backward(api):
    """hdf_backward_after_apply takes the range maps, coefficients,
    denominators and guard list that the last apply left in the handle and
    gives the gradients of hdf_backward bit for bit (no pixel here needs the
    FP64 recomputation); it refuses when the handle's last call was not an
    apply, and the autograd function uses it."""
    f = synthetic.color_rectangles(70, 45, seed=97)
    f = np.clip(f + np.random.default_rng(98).normal(0, 0.03, f.shape), 0, 1).astype(np.float32)
    fd = torch.from_numpy(f).cuda()
    G = torch.from_numpy(np.random.default_rng(99).normal(size=f.shape).astype(np.float32)).cuda()
    flt = api.HDFilter(70, 45, 3, 3, 8, 2.0, 0.3)
    flt.cluster(fd)
    gf0, gs0, gr0 = flt.backward(fd, fd, G)
    g = flt.apply(fd, fd)
    gf1, gs1, gr1 = flt.backward(fd, fd, G, g=g)
    assert torch.equal(gf0, gf1)
    assert float(gs0) == float(gs1) and float(gr0) == float(gr1)
    assert flt.stats()["rescued_pixels"] == 0
    with pytest.raises(Exception):      # the backward ended the apply's state
        flt.backward(fd, fd, G, g=g)
    g = flt.apply(fd, fd)
    flt.cluster(fd)
    with pytest.raises(Exception):      # so does a clustering
        flt.backward(fd, fd, G, g=g)
    # autograd: forward then backward on the same handle takes the shortcut
    fx = fd.clone().requires_grad_(True)
    ls = torch.tensor(math.log(2.0), device="cuda", requires_grad=True)
    lr = torch.tensor(math.log(0.3), device="cuda", requires_grad=True)
    out = api.fast_filter(fx, ls, lr, flt)
    seq = flt._seq
    (out * G).sum().backward()
    assert flt._seq == seq + 1
    gf2, gs2, gr2 = flt.backward(fd, fd, G)
    assert torch.equal(fx.grad, gf2)
