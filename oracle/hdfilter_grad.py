"""FP64 reference gradients of the fast filter (Algorithm 1, Eq. (15)-(16)).

TEST INFRASTRUCTURE.  Used only by the tests to check the CUDA backward pass.

A second, independent implementation of the approximation written with
PyTorch CPU float64 tensors, differentiated by autograd, with the centres mu
and the window half-width S held fixed and sigma_s, sigma_r entering as
exp(log sigma).  It is pinned in tests/test_oracle_grad.py against central
finite differences of the numpy oracle (oracle/hdfilter_oracle.py), so a
mistake in either implementation shows.

Gradients are defined where the denominator guard does not fire (the tests
use inputs without guarded pixels) and for a full-rank A, where
A^+ = A^{-1} (Eq. (11)); the derivative of a truncated pseudo-inverse is not
defined.
"""
from __future__ import annotations

import math

import torch


def _window_1d(log_sigma_s: torch.Tensor, S: int) -> torch.Tensor:
    t = torch.arange(-S, S + 1, dtype=torch.float64)
    sig = torch.exp(log_sigma_s)
    return torch.exp(-(t * t) / (2.0 * sig * sig))


def _conv_rows(x: torch.Tensor, w: torch.Tensor) -> torch.Tensor:
    """out[..., c] = sum_t w[t] x[..., c - t], zero outside the image."""
    S = (w.numel() - 1) // 2
    Wd = x.shape[-1]
    out = torch.zeros_like(x)
    for t in range(-S, S + 1):
        c0, c1 = max(0, t), min(Wd, Wd + t)
        if c0 < c1:
            out[..., c0:c1] = out[..., c0:c1] + w[t + S] * x[..., c0 - t:c1 - t]
    return out


def _conv2(x: torch.Tensor, w: torch.Tensor) -> torch.Tensor:
    y = _conv_rows(x, w)
    return _conv_rows(y.transpose(-1, -2), w).transpose(-1, -2)


def fast_filter_torch(f: torch.Tensor, p: torch.Tensor | None, mu: torch.Tensor,
                      log_sigma_s: torch.Tensor, log_sigma_r: torch.Tensor, S: int) -> torch.Tensor:
    """Algorithm 1 in float64 torch: b_k = phi(mu_k - p), c = A^{-1} b,
    g = sum_k c_k (omega * (b_k f)) / sum_k c_k (omega * b_k).  p=None: p = f."""
    p = f if p is None else p
    sr = torch.exp(log_sigma_r)
    d2 = ((p[None, :, :, :] - mu[:, :, None, None]) ** 2).sum(dim=1)          # (K, H, W)
    B = torch.exp(-d2 / (2.0 * sr * sr))
    dmu = ((mu[:, None, :] - mu[None, :, :]) ** 2).sum(dim=2)
    A = torch.exp(-dmu / (2.0 * sr * sr))
    K = mu.shape[0]
    C = torch.linalg.solve(A, B.reshape(K, -1)).reshape(B.shape)              # A^{-1} b(i)
    w = _window_1d(log_sigma_s, S)
    num = torch.zeros_like(f)
    den = torch.zeros_like(f[0])
    for k in range(K):
        num = num + C[k] * _conv2(B[k][None] * f, w)
        den = den + C[k] * _conv2(B[k], w)
    return num / den


def grads(f, p, mu, sigma_s: float, sigma_r: float, S: int, G):
    """dL/df, dL/dlog sigma_s, dL/dlog sigma_r for L = <G, g_hat> (float64).
    p=None means guide = image (the gradient then includes the guide path)."""
    f = torch.tensor(f, dtype=torch.float64, requires_grad=True)
    pt = None if p is None else torch.tensor(p, dtype=torch.float64)
    mu = torch.tensor(mu, dtype=torch.float64)
    ls = torch.tensor(float(torch.log(torch.tensor(sigma_s, dtype=torch.float64))),
                      dtype=torch.float64, requires_grad=True)
    lr = torch.tensor(float(torch.log(torch.tensor(sigma_r, dtype=torch.float64))),
                      dtype=torch.float64, requires_grad=True)
    g = fast_filter_torch(f, pt, mu, ls, lr, S)
    L = (g * torch.tensor(G, dtype=torch.float64)).sum()
    L.backward()
    return f.grad.numpy(), float(ls.grad), float(lr.grad), g.detach().numpy()


def bruteforce_torch(f: torch.Tensor, p: torch.Tensor | None, log_sigma_s: torch.Tensor,
                     log_sigma_r: torch.Tensor, S: int) -> torch.Tensor:
    """Eq. (1)-(2) in float64 torch, differentiable in f, log sigma_s and log
    sigma_r: g(i) = sum_j omega(j) phi(p(i-j) - p(i)) f(i-j) / eta(i) over
    W = [-S, S]^2, neighbours outside the image left out.  p=None: p = f."""
    p = f if p is None else p
    n, H, W = f.shape
    ss, sr = torch.exp(log_sigma_s), torch.exp(log_sigma_r)
    num = torch.zeros_like(f)
    den = torch.zeros_like(f[0])
    for j1 in range(-S, S + 1):
        for j2 in range(-S, S + 1):
            y0, y1 = max(0, j1), min(H, H + j1)
            x0, x1 = max(0, j2), min(W, W + j2)
            if y0 >= y1 or x0 >= x1:
                continue
            w = torch.exp(-torch.tensor(float(j1 * j1 + j2 * j2), dtype=torch.float64)
                          / (2.0 * ss * ss))
            pi = p[:, y0:y1, x0:x1]
            pn = p[:, y0 - j1:y1 - j1, x0 - j2:x1 - j2]
            wt = w * torch.exp(-((pn - pi) ** 2).sum(dim=0) / (2.0 * sr * sr))
            pad = (x0, W - x1, y0, H - y1)
            num = num + torch.nn.functional.pad(wt * f[:, y0 - j1:y1 - j1, x0 - j2:x1 - j2], pad)
            den = den + torch.nn.functional.pad(wt, pad)
    return num / den


def brute_grads(f, p, sigma_s: float, sigma_r: float, S: int, G):
    """dL/df, dL/dlog sigma_s, dL/dlog sigma_r of L = <G, g> for the brute
    force (float64 autograd); p=None means guide = image."""
    f = torch.tensor(f, dtype=torch.float64, requires_grad=True)
    pt = None if p is None else torch.tensor(p, dtype=torch.float64)
    ls = torch.tensor(math.log(sigma_s), dtype=torch.float64, requires_grad=True)
    lr = torch.tensor(math.log(sigma_r), dtype=torch.float64, requires_grad=True)
    g = bruteforce_torch(f, pt, ls, lr, S)
    (g * torch.tensor(G, dtype=torch.float64)).sum().backward()
    return f.grad.numpy(), float(ls.grad), float(lr.grad), g.detach().numpy()
