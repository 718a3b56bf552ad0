"""Seeded synthetic inputs for the fast high-dimensional bilateral / NLM filter.

These generators stand in for the paper's image datasets (Kodak, hyperspectral
cubes, natural grayscale images), which are not available.  They produce
planar float32 arrays shaped (channels, H, W) with values of the same scale and
structure as the paper's workloads (Sec. III): piecewise-constant colour scenes
for colour bilateral filtering, smooth spectral mixtures for hyperspectral
filtering, and a smooth field with edges for nonlocal means.

This module holds no arithmetic of the filter itself: it is shared by the CPU
oracle tests, the GPU parity tests and the benchmark only as a source of
inputs.  All randomness comes from ``numpy.random.default_rng(seed)``.
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np


def color_rectangles(H: int, W: int, n_rect: int = 12, noise: float = 0.05,
                     seed: int = 0, channels: int = 3) -> np.ndarray:
    """Background colour plus ``n_rect`` axis-aligned constant-colour rectangles
    painted in order, plus i.i.d. Gaussian noise, clipped to [0, 1].

    Returns float32 (channels, H, W)."""
    rng = np.random.default_rng(seed)
    img = np.empty((channels, H, W), dtype=np.float64)
    img[:] = rng.uniform(0.0, 1.0, size=(channels, 1, 1))
    for _ in range(n_rect):
        y0, y1 = np.sort(rng.integers(0, H, size=2))
        x0, x1 = np.sort(rng.integers(0, W, size=2))
        col = rng.uniform(0.0, 1.0, size=(channels, 1, 1))
        img[:, y0:y1 + 1, x0:x1 + 1] = col
    img += rng.normal(0.0, noise, size=img.shape)
    np.clip(img, 0.0, 1.0, out=img)
    return img.astype(np.float32)


def smooth_spectra(bands: int, n_end: int, rng: np.random.Generator) -> np.ndarray:
    """``n_end`` smooth spectra over the band index, each a sum of three
    Gaussian bumps (amplitude U[0.2,1], centre U[0,bands-1], width U[2,8]),
    scaled so that its maximum is 1.  Returns float64 (n_end, bands)."""
    b = np.arange(bands, dtype=np.float64)
    out = np.zeros((n_end, bands))
    for e in range(n_end):
        for _ in range(3):
            amp = rng.uniform(0.2, 1.0)
            cen = rng.uniform(0.0, bands - 1.0)
            wid = rng.uniform(2.0, 8.0)
            out[e] += amp * np.exp(-0.5 * ((b - cen) / wid) ** 2)
        out[e] /= out[e].max()
    return out


def hyperspectral_mixture(H: int, W: int, bands: int = 31, n_end: int = 6,
                          alpha: float = 0.5, noise: float = 0.02,
                          seed: int = 1) -> np.ndarray:
    """Each pixel is a convex combination (Dirichlet(alpha) abundances, i.i.d.
    per pixel) of ``n_end`` smooth spectra, plus Gaussian noise.

    Returns float32 (bands, H, W)."""
    rng = np.random.default_rng(seed)
    spectra = smooth_spectra(bands, n_end, rng)
    ab = rng.dirichlet(alpha * np.ones(n_end), size=H * W)          # (HW, n_end)
    cube = (ab @ spectra).T.reshape(bands, H, W)
    cube = cube + rng.normal(0.0, noise, size=cube.shape)
    return cube.astype(np.float32)


def _lowpass_wrap(x: np.ndarray, sigma: float) -> np.ndarray:
    """Periodic Gaussian low-pass of a 2-D array through the FFT (input
    synthesis only)."""
    H, W = x.shape
    fy = np.fft.fftfreq(H)[:, None]
    fx = np.fft.fftfreq(W)[None, :]
    tf = np.exp(-2.0 * (math.pi * sigma) ** 2 * (fy * fy + fx * fx))
    return np.real(np.fft.ifft2(np.fft.fft2(x) * tf))


def smooth_field_with_edges(H: int, W: int, noise: float = 0.1, n_edges: int = 8,
                            seed: int = 2) -> np.ndarray:
    """Grayscale test image for nonlocal means: uniform noise low-pass filtered
    (Gaussian, 16 px), rescaled to [0.2, 0.8], plus ``n_edges`` random
    half-plane steps of +-0.2, plus i.i.d. Gaussian noise of std ``noise``.

    Returns float32 (1, H, W)."""
    rng = np.random.default_rng(seed)
    field = _lowpass_wrap(rng.uniform(0.0, 1.0, size=(H, W)), 16.0)
    lo, hi = field.min(), field.max()
    field = 0.2 + 0.6 * (field - lo) / max(hi - lo, 1e-12)
    yy, xx = np.mgrid[0:H, 0:W].astype(np.float64)
    for _ in range(n_edges):
        theta = rng.uniform(0.0, 2.0 * math.pi)
        cy, cx = rng.uniform(0, H), rng.uniform(0, W)
        step = 0.2 if rng.uniform() < 0.5 else -0.2
        side = (np.cos(theta) * (xx - cx) + np.sin(theta) * (yy - cy)) > 0
        field = field + step * side
    field = field + rng.normal(0.0, noise, size=field.shape)
    return field[None].astype(np.float32)


def lowlight_infrared(H: int, W: int, seed: int = 5) -> tuple[np.ndarray, np.ndarray]:
    """A dark, noisy grayscale frame and a registered infrared frame of the
    same scene (stand-in for the low-light + infrared pair of Sec. III-E):
    the scene is ``smooth_field_with_edges`` without noise; the low-light
    frame is 0.15 x scene + N(0, 0.02^2) noise; the infrared frame is
    0.6 x scene + 0.2 x an independent smooth texture (low-pass 8 px) +
    N(0, 0.005^2) noise, clipped to [0, 1].  Returns two float32 (1, H, W)."""
    rng = np.random.default_rng(seed)
    scene = smooth_field_with_edges(H, W, noise=0.0, seed=seed + 1000)[0].astype(np.float64)
    dark = 0.15 * scene + rng.normal(0.0, 0.02, size=(H, W))
    tex = _lowpass_wrap(rng.uniform(0.0, 1.0, size=(H, W)), 8.0)
    tex = (tex - tex.min()) / max(tex.max() - tex.min(), 1e-12)
    ir = np.clip(0.6 * scene + 0.2 * tex + rng.normal(0.0, 0.005, size=(H, W)), 0.0, 1.0)
    return dark[None].astype(np.float32), ir[None].astype(np.float32)


@dataclasses.dataclass
class BatchItem:
    """One image of the batched serving workload with its filter parameters."""
    image: np.ndarray      # float32 (n, H, W)
    sigma_s: float
    sigma_r: float
    K: int


def serving_batch(count: int = 64, seed: int = 4,
                  sides=(256, 512, 1024, 2048)) -> list[BatchItem]:
    """Mixed batch: image sides uniform over ``sides``; the first half RGB
    rectangles scenes, the second half 16-band spectral mixtures;
    sigma_s ~ U[2, 8], sigma_r ~ U[0.1, 0.3], K uniform over {8, 16, 32}."""
    rng = np.random.default_rng(seed)
    items = []
    for b in range(count):
        side = int(rng.choice(sides))
        sub = int(rng.integers(0, 2**31 - 1))
        if b < count // 2:
            img = color_rectangles(side, side, seed=sub)
        else:
            img = hyperspectral_mixture(side, side, bands=16, seed=sub)
        items.append(BatchItem(img, float(rng.uniform(2.0, 8.0)),
                               float(rng.uniform(0.1, 0.3)),
                               int(rng.choice([8, 16, 32]))))
    return items


# Named workloads with the sizes the benchmark and tests use.
def workload(name: str) -> dict:
    """Return the inputs and parameters of a named workload.

    ``color256``      3x256x256 rectangles, sigma_s=3, sigma_r=0.2, K=8.
    ``hyper512``      31x512x512 spectral mixture, sigma_s=5, sigma_r=0.3, K=32.
    ``nlm1024``       1x1024x1024 smooth field + edges (guide: 7x7 patches
                      reduced to 6 PCA features), sigma_s=5, sigma_r=0.15, K=32.
    ``color2048``     3x2048x2048 rectangles, sigma_s=8, sigma_r=0.15, K=16.
    """
    if name == "color256":
        return dict(f=color_rectangles(256, 256, seed=0), sigma_s=3.0, sigma_r=0.2, K=8)
    if name == "hyper512":
        return dict(f=hyperspectral_mixture(512, 512, bands=31, seed=1),
                    sigma_s=5.0, sigma_r=0.3, K=32)
    if name == "nlm1024":
        return dict(f=smooth_field_with_edges(1024, 1024, seed=2),
                    sigma_s=5.0, sigma_r=0.15, K=32, patch=7, pca_dims=6)
    if name == "color2048":
        return dict(f=color_rectangles(2048, 2048, seed=3), sigma_s=8.0, sigma_r=0.15, K=16)
    raise KeyError(name)
