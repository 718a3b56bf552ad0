"""Pin the FP64 gradient reference (torch autograd through an independent
implementation of Algorithm 1) against central finite differences of the
numpy oracle, and its forward against the numpy oracle.  CPU only."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import hdfilter_grad as OG
from oracle import hdfilter_oracle as O
from paper_1811_02363_gb300 import synthetic


def _case(separate):
    f = synthetic.color_rectangles(14, 12, seed=71).astype(np.float64)
    rng = np.random.default_rng(72)
    f = np.clip(f + 0.05 * rng.normal(size=f.shape), 0, 1)
    p = None
    if separate:
        p = rng.uniform(size=(2, 14, 12))
    guide = f if p is None else p
    mu, _, _ = O.bisecting_kmeans(guide.reshape(guide.shape[0], -1).T, 5)
    G = rng.normal(size=f.shape)
    return f, p, mu, G


@pytest.mark.parametrize("separate", [False, True])
def test_torch_forward_matches_numpy_oracle(separate):
    f, p, mu, G = _case(separate)
    _, _, _, g = OG.grads(f, p, mu, 1.3, 0.35, 3, G)
    ref = O.fast_filter(f, f if p is None else p, mu, 1.3, 0.35, 3, guard=False)
    assert np.max(np.abs(g - ref)) < 1e-12


@pytest.mark.parametrize("separate", [False, True])
def test_gradients_match_central_differences(separate):
    f, p, mu, G = _case(separate)
    ss, sr, S = 1.3, 0.35, 3
    gf, gls, glr, _ = OG.grads(f, p, mu, ss, sr, S, G)

    def L(ff, s_s, s_r):
        return float((O.fast_filter(ff, ff if p is None else p, mu, s_s, s_r, S, guard=False) * G).sum())

    h = 1e-5
    # sigma derivatives in log space
    d_ls = (L(f, ss * math.exp(h), sr) - L(f, ss * math.exp(-h), sr)) / (2 * h)
    d_lr = (L(f, ss, sr * math.exp(h)) - L(f, ss, sr * math.exp(-h))) / (2 * h)
    assert abs(d_ls - gls) <= 1e-6 * max(1.0, abs(d_ls))
    assert abs(d_lr - glr) <= 1e-6 * max(1.0, abs(d_lr))
    # image derivative at a few entries (including border pixels)
    for idx in [(0, 0, 0), (1, 7, 5), (2, 13, 11), (0, 3, 9)]:
        fp, fm = f.copy(), f.copy()
        fp[idx] += h
        fm[idx] -= h
        d = (L(fp, ss, sr) - L(fm, ss, sr)) / (2 * h)
        assert abs(d - gf[idx]) <= 1e-6 * max(1.0, abs(d)), (idx, d, gf[idx])
