"""Python surface of the GB300 fast high-dimensional bilateral / NLM filter.

Thin wrappers over the C ABI (include/hdfilter.h): they check tensor shapes,
dtypes and devices, pass raw pointers and torch's current CUDA stream, and
raise on error codes.  PyTorch supplies device memory and streams only; all
arithmetic runs in libhdfilter's kernels, and there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import math

import numpy as np
import torch

from . import _lib as L


def _stream() -> C.c_void_p:
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t: torch.Tensor) -> C.c_void_p:
    return C.c_void_p(t.data_ptr())


def _check_image(t: torch.Tensor, name: str, dtype=torch.float32) -> None:
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous (planar C x H x W)")
    if t.dim() != 3:
        raise ValueError(f"{name} must be (C, H, W)")


def window_halfwidth(sigma_s: float) -> int:
    """S = ceil(3 sigma_s) (Sec. III)."""
    return int(math.ceil(3.0 * sigma_s))


def make_desc(H, W, n, rho, K, sigma_s, sigma_r, S=0, guide_dtype="f32", coef="opt",
              spatial="gauss") -> L.hdf_desc:
    d = L.hdf_desc()
    d.H, d.W, d.n, d.rho, d.K = int(H), int(W), int(n), int(rho), int(K)
    d.S = int(S) if S else window_halfwidth(sigma_s)
    d.sigma_s, d.sigma_r = float(sigma_s), float(sigma_r)
    d.guide_dtype = {"f32": L.HDF_GUIDE_F32, "bf16": L.HDF_GUIDE_BF16}[guide_dtype]
    d.coef = {"opt": L.HDF_COEF_OPT, "indicator": L.HDF_COEF_INDICATOR}[coef]
    d.spatial = {"gauss": L.HDF_SPATIAL_GAUSS, "box": L.HDF_SPATIAL_BOX,
                 "young": L.HDF_SPATIAL_YOUNG}[spatial]
    return d


class HDFilter:
    """One filter instance (Algorithm 1) for images of a fixed shape.

    ``cluster(p)`` runs bisecting K-means + the FP64 pseudo-inverse on the
    device; ``set_centers(mu)`` installs given centres instead; ``apply(f, p)``
    filters; ``backward(...)`` returns gradients."""

    def __init__(self, H, W, n, rho, K, sigma_s, sigma_r, S=0, guide_dtype="f32", coef="opt",
                 spatial="gauss"):
        self.desc = make_desc(H, W, n, rho, K, sigma_s, sigma_r, S, guide_dtype, coef, spatial)
        self._h = C.c_void_p()
        L.check(L.lib().hdf_create(C.byref(self._h), C.byref(self.desc)), "hdf_create")
        L.check(L.lib().hdf_get_desc(self._h, C.byref(self.desc)), "hdf_get_desc")
        self.guide_torch_dtype = torch.float32 if guide_dtype == "f32" else torch.bfloat16
        self._seq = 0   # calls that change the handle's state (apply, cluster, backward, ...)

    # -- lifecycle
    def close(self) -> None:
        if self._h:
            L.lib().hdf_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def S(self) -> int:
        return self.desc.S

    def _check_guide(self, p: torch.Tensor) -> None:
        _check_image(p, "p", self.guide_torch_dtype)
        if tuple(p.shape) != (self.desc.rho, self.desc.H, self.desc.W):
            raise ValueError(f"guide shape {tuple(p.shape)} != (rho, H, W)")

    def _check_f(self, f: torch.Tensor, name="f") -> None:
        _check_image(f, name)
        if tuple(f.shape) != (self.desc.n, self.desc.H, self.desc.W):
            raise ValueError(f"{name} shape {tuple(f.shape)} != (n, H, W)")

    # -- Algorithm 1 steps
    def cluster(self, p: torch.Tensor) -> None:
        self._check_guide(p)
        L.check(L.lib().hdf_cluster(self._h, _ptr(p), _stream()), "hdf_cluster")
        self._seq += 1

    def set_centers(self, mu) -> None:
        mu = np.ascontiguousarray(np.asarray(mu, dtype=np.float32))
        if mu.ndim != 2 or mu.shape[1] != self.desc.rho:
            raise ValueError("centres must be (K, rho)")
        self._mu_keepalive = mu
        L.check(L.lib().hdf_set_centers(self._h, mu.ctypes.data_as(C.c_void_p), mu.shape[0],
                                        _stream()), "hdf_set_centers")
        self._seq += 1
        torch.cuda.current_stream().synchronize()

    def get_centers(self) -> np.ndarray:
        out = np.zeros((self.desc.K, self.desc.rho), dtype=np.float32)
        k = C.c_int()
        L.check(L.lib().hdf_get_centers(self._h, out.ctypes.data_as(C.c_void_p), C.byref(k),
                                        _stream()), "hdf_get_centers")
        return out[:k.value].copy()

    def get_pinv(self) -> np.ndarray:
        out = np.zeros(self.desc.K * self.desc.K, dtype=np.float64)
        L.check(L.lib().hdf_get_pinv(self._h, out.ctypes.data_as(C.c_void_p), _stream()),
                "hdf_get_pinv")
        k = self.stats()["K_eff"]
        return out[:k * k].reshape(k, k)

    def get_labels(self) -> torch.Tensor:
        lab = torch.empty(self.desc.H * self.desc.W, dtype=torch.int32, device="cuda")
        L.check(L.lib().hdf_get_labels(self._h, _ptr(lab), _stream()), "hdf_get_labels")
        return lab

    def apply(self, f: torch.Tensor, p: torch.Tensor | None = None,
              out: torch.Tensor | None = None) -> torch.Tensor:
        self._check_f(f)
        p = f if p is None else p
        self._check_guide(p)
        g = torch.empty_like(f) if out is None else out
        self._check_f(g, "out")
        L.check(L.lib().hdf_apply(self._h, _ptr(f), _ptr(p), _ptr(g), _stream()), "hdf_apply")
        self._seq += 1
        return g

    def backward(self, f: torch.Tensor, p: torch.Tensor, grad_g: torch.Tensor,
                 g: torch.Tensor | None = None):
        """Returns (dL/df, dL/dlog sigma_s, dL/dlog sigma_r) as CUDA tensors.
        With ``g`` (the output of the last ``apply`` of this filter, from the
        same f and p) the forward state left by that apply is reused
        (hdf_backward_after_apply) instead of recomputed."""
        self._check_f(f)
        self._check_guide(p)
        self._check_f(grad_g, "grad_g")
        gf = torch.empty_like(f)
        gs = torch.zeros(2, dtype=torch.float64, device=f.device)
        if g is None:
            L.check(L.lib().hdf_backward(self._h, _ptr(f), _ptr(p), _ptr(grad_g), _ptr(gf),
                                         _ptr(gs), _stream()), "hdf_backward")
        else:
            self._check_f(g, "g")
            L.check(L.lib().hdf_backward_after_apply(self._h, _ptr(f), _ptr(p), _ptr(g),
                                                     _ptr(grad_g), _ptr(gf), _ptr(gs), _stream()),
                    "hdf_backward_after_apply")
        self._seq += 1
        return gf, gs[0], gs[1]

    def set_sigmas(self, sigma_s: float, sigma_r: float) -> None:
        """New sigma_s and sigma_r for the following calls (hdf_set_sigmas:
        S, the centres and the buffers stay; A^+ is refitted on the device)."""
        L.check(L.lib().hdf_set_sigmas(self._h, float(sigma_s), float(sigma_r), _stream()),
                "hdf_set_sigmas")
        self._seq += 1
        self.desc.sigma_s, self.desc.sigma_r = float(sigma_s), float(sigma_r)

    def _use_sigmas(self, sigma_s: float, sigma_r: float) -> None:
        if sigma_s != self.desc.sigma_s or sigma_r != self.desc.sigma_r:
            self.set_sigmas(sigma_s, sigma_r)

    def nlm_guide(self, f: torch.Tensor, patch: int = 7, out: torch.Tensor | None = None) -> torch.Tensor:
        """PCA-reduced patch guide (desc.rho features) of the image f (n, H, W)."""
        self._check_f(f)
        p = out if out is not None else torch.empty((self.desc.rho, self.desc.H, self.desc.W),
                                                    dtype=torch.float32, device=f.device)
        L.check(L.lib().hdf_nlm_guide(self._h, _ptr(f), int(patch), _ptr(p), _stream()),
                "hdf_nlm_guide")
        return p

    def trace(self, cap: int = 2048) -> np.ndarray:
        """(phase, ns) events of the last clustering (see hdf_get_trace)."""
        buf = np.zeros(2 * cap, dtype=np.int64)
        n = C.c_int()
        L.check(L.lib().hdf_get_trace(self._h, buf.ctypes.data_as(C.c_void_p), cap, C.byref(n),
                                      _stream()), "hdf_get_trace")
        return buf[:2 * n.value].reshape(-1, 2)

    def set_stage_timing(self, on: bool = True) -> None:
        """Record CUDA events between the stages of every following apply."""
        L.check(L.lib().hdf_set_stage_timing(self._h, 1 if on else 0), "hdf_set_stage_timing")

    def stage_times(self) -> dict:
        """ms of the last timed apply: range maps, tile kernel, the rest."""
        arr = (C.c_float * 3)()
        cnt = C.c_int()
        L.check(L.lib().hdf_get_stage_times(self._h, arr, 3, C.byref(cnt)), "hdf_get_stage_times")
        names = ["rangemap", "tile", "rest"]
        return {names[i]: float(arr[i]) for i in range(cnt.value)}

    def set_wait_limit(self, seconds: float) -> None:
        """Limit of each device-side wait of ``cluster`` (default 2 s)."""
        L.check(L.lib().hdf_set_wait_limit(self._h, float(seconds)), "hdf_set_wait_limit")

    def stats(self) -> dict:
        s = L.hdf_stats()
        code = L.lib().hdf_get_stats(self._h, C.byref(s), _stream())
        d = {k: getattr(s, k) for k, _ in L.hdf_stats._fields_}
        if code != L.HDF_OK:
            raise L.HDFError(code, "device status")
        return d


def scale_guide(p: torch.Tensor, sigma_r, out: torch.Tensor | None = None) -> torch.Tensor:
    """The guide divided by sigma_r per dimension (hdf_scale_guide): with it
    and sigma_r = 1 every filter call uses the anisotropic range kernel
    exp(-sum_d x_d^2 / (2 sigma_r[d]^2)) of Sec. III-E."""
    if not p.is_cuda or p.dim() != 3 or not p.is_contiguous():
        raise ValueError("p must be a contiguous CUDA (rho, H, W) tensor")
    if p.dtype not in (torch.float32, torch.bfloat16):
        raise ValueError("p must be float32 or bfloat16")
    rho, H, W = p.shape
    sr = np.ascontiguousarray(np.broadcast_to(np.asarray(sigma_r, dtype=np.float64), (rho,)))
    q = torch.empty((rho, H, W), dtype=torch.float32, device=p.device) if out is None else out
    _check_image(q, "out")
    gd = L.HDF_GUIDE_F32 if p.dtype == torch.float32 else L.HDF_GUIDE_BF16
    L.check(L.lib().hdf_scale_guide(_ptr(p), gd, rho, H, W, sr.ctypes.data_as(C.c_void_p), _ptr(q),
                                    _stream()), "hdf_scale_guide")
    return q


def probe_peaks() -> tuple[float, float]:
    """Measured FP32 and FP64 FMA peak rates of the current GPU, TFLOP/s."""
    a, b = C.c_double(), C.c_double()
    L.check(L.lib().hdf_probe_peaks(C.byref(a), C.byref(b), _stream()), "hdf_probe_peaks")
    return a.value, b.value


def bruteforce(f: torch.Tensor, p: torch.Tensor | None, sigma_s: float, sigma_r: float,
               S: int = 0, out: torch.Tensor | None = None, spatial: str = "gauss") -> torch.Tensor:
    """Eq. (1)-(2) by direct summation on the GPU."""
    _check_image(f, "f")
    p = f if p is None else p
    if not p.is_cuda or p.dim() != 3 or not p.is_contiguous():
        raise ValueError("p must be a contiguous CUDA (rho, H, W) tensor")
    if p.dtype not in (torch.float32, torch.bfloat16):
        raise ValueError("p must be float32 or bfloat16")
    n, H, W = f.shape
    d = make_desc(H, W, n, p.shape[0], 1, sigma_s, sigma_r, S,
                  "f32" if p.dtype == torch.float32 else "bf16", spatial=spatial)
    g = torch.empty_like(f) if out is None else out
    _check_image(g, "out")
    L.check(L.lib().hdf_bruteforce(C.byref(d), _ptr(f), _ptr(p), _ptr(g), _stream()),
            "hdf_bruteforce")
    return g


class _FastFilterFn(torch.autograd.Function):
    """g = fast filter of f (guide = f or a fixed separate guide); gradients
    for f, log sigma_s and log sigma_r from hdf_backward (centres and S fixed)."""

    @staticmethod
    def forward(ctx, f, log_sigma_s, log_sigma_r, flt, guide):
        ctx.sigmas = (math.exp(float(log_sigma_s)), math.exp(float(log_sigma_r)))
        ctx.dtypes = (log_sigma_s.dtype, log_sigma_r.dtype)
        flt._use_sigmas(*ctx.sigmas)
        p = f if guide is None else guide
        g = flt.apply(f.contiguous(), p)
        ctx.flt = flt
        ctx.guide = guide
        ctx.seq = flt._seq          # the handle still holds this apply's state while unchanged
        ctx.save_for_backward(f, g)
        return g

    @staticmethod
    def backward(ctx, grad_g):
        f, g = ctx.saved_tensors
        p = f if ctx.guide is None else ctx.guide
        ctx.flt._use_sigmas(*ctx.sigmas)    # the widths of this forward call
        reuse = g if ctx.flt._seq == ctx.seq else None
        gf, gls, glr = ctx.flt.backward(f.contiguous(), p, grad_g.contiguous(), g=reuse)
        return gf, gls.to(ctx.dtypes[0]), glr.to(ctx.dtypes[1]), None, None


def fast_filter(f: torch.Tensor, log_sigma_s: torch.Tensor, log_sigma_r: torch.Tensor,
                flt: HDFilter, guide: torch.Tensor | None = None) -> torch.Tensor:
    """Differentiable fast filter (Algorithm 1) with the centres installed in
    ``flt``.  The widths exp(log_sigma_s), exp(log_sigma_r) are live: a call
    whose values differ from the handle's installs them (hdf_set_sigmas: S
    and the centres stay, A^+ is refitted), so their gradients can drive an
    optimisation of the widths; gradients flow to f, log_sigma_s and
    log_sigma_r."""
    return _FastFilterFn.apply(f, log_sigma_s, log_sigma_r, flt, guide)


class Batch:
    """Many images through Algorithm 1 together (hdf_batch_*): one launch per
    stage for the whole batch, one persistent launch for all convolution /
    combine tiles, CUDA-graph replay, and an autotuner for tile shapes.

    ``specs``: one dict per image with keys H, W, n, K, sigma_s, sigma_r and
    optionally rho (default n), S, guide_dtype ("f32" / "bf16"), coef, spatial
    ("gauss" / "box").
    ``bind(fs, gs, ps=None)`` binds CUDA tensors (ps entries None = guide is
    the image; with guide_dtype "bf16" the run stores it as bfloat16)."""

    def __init__(self, specs):
        self.specs = [dict(s) for s in specs]
        descs = (L.hdf_desc * len(specs))()
        for i, s in enumerate(self.specs):
            descs[i] = make_desc(s["H"], s["W"], s["n"], s.get("rho", s["n"]), s["K"],
                                 s["sigma_s"], s["sigma_r"], s.get("S", 0),
                                 s.get("guide_dtype", "f32"), s.get("coef", "opt"),
                                 s.get("spatial", "gauss"))
        self.descs = descs
        self._b = C.c_void_p()
        L.check(L.lib().hdf_batch_create(C.byref(self._b), len(specs), descs), "hdf_batch_create")
        self._bound = None

    def close(self) -> None:
        if self._b:
            L.lib().hdf_batch_destroy(self._b)
            self._b = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __len__(self) -> int:
        return len(self.specs)

    def bind(self, fs, gs, ps=None) -> None:
        n = len(self.specs)
        if len(fs) != n or len(gs) != n or (ps is not None and len(ps) != n):
            raise ValueError("one tensor per image")
        for i, (f, g) in enumerate(zip(fs, gs)):
            d = self.descs[i]
            _check_image(f, f"f[{i}]")
            _check_image(g, f"g[{i}]")
            if tuple(f.shape) != (d.n, d.H, d.W) or tuple(g.shape) != (d.n, d.H, d.W):
                raise ValueError(f"image {i}: expected ({d.n}, {d.H}, {d.W})")
            p = None if ps is None else ps[i]
            if p is not None:
                want = torch.float32 if d.guide_dtype == L.HDF_GUIDE_F32 else torch.bfloat16
                _check_image(p, f"p[{i}]", want)
                if tuple(p.shape) != (d.rho, d.H, d.W):
                    raise ValueError(f"guide {i}: expected ({d.rho}, {d.H}, {d.W})")
        arr = C.c_void_p * n
        fa = arr(*[f.data_ptr() for f in fs])
        ga = arr(*[g.data_ptr() for g in gs])
        pa = arr(*[(0 if ps is None or ps[i] is None else ps[i].data_ptr()) for i in range(n)])
        L.check(L.lib().hdf_batch_bind(self._b, fa, pa, ga), "hdf_batch_bind")
        self._bound = (list(fs), list(gs), None if ps is None else list(ps))   # keep alive

    def set_centers(self, i: int, mu) -> None:
        d = self.descs[i]
        mu = np.ascontiguousarray(np.asarray(mu, dtype=np.float32))
        if mu.ndim != 2 or mu.shape[1] != d.rho:
            raise ValueError("centres must be (K, rho)")
        L.check(L.lib().hdf_batch_set_centers(self._b, int(i), mu.ctypes.data_as(C.c_void_p),
                                              mu.shape[0]), "hdf_batch_set_centers")

    def run(self, graph: bool = True, timed: bool = False, skip_cluster: bool = False) -> None:
        flags = (L.HDF_BATCH_GRAPH if graph else 0) | (L.HDF_BATCH_TIMED if timed else 0) | \
            (L.HDF_BATCH_SKIP_CLUSTER if skip_cluster else 0)
        L.check(L.lib().hdf_batch_run(self._b, flags, _stream()), "hdf_batch_run")

    def tune(self, reps: int = 3) -> list[dict]:
        L.check(L.lib().hdf_batch_tune(self._b, int(reps), _stream()), "hdf_batch_tune")
        return self.tuning()

    def tuning(self) -> list[dict]:
        cnt = C.c_int()
        L.check(L.lib().hdf_batch_get_tuning(self._b, None, 0, C.byref(cnt)), "get_tuning")
        arr = (L.hdf_tile_trial * max(1, cnt.value))()
        L.check(L.lib().hdf_batch_get_tuning(self._b, arr, cnt.value, C.byref(cnt)), "get_tuning")
        return [{k: getattr(arr[i], k) for k, _ in L.hdf_tile_trial._fields_}
                for i in range(cnt.value)]

    def set_shape(self, SB: int, planes: int, P: int, TY: int) -> None:
        L.check(L.lib().hdf_batch_set_shape(self._b, SB, planes, P, TY), "hdf_batch_set_shape")

    def times(self) -> list[float]:
        """Stage times (ms) of the last timed run: reset, bf16 guides,
        clustering, fit, range maps, persistent tiles, normalise."""
        arr = (C.c_float * 7)()
        cnt = C.c_int()
        L.check(L.lib().hdf_batch_get_times(self._b, arr, 7, C.byref(cnt)), "get_times")
        return [arr[i] for i in range(cnt.value)]

    def get_centers(self, i: int) -> np.ndarray:
        d = self.descs[i]
        mu = np.zeros((d.K, d.rho), np.float32)
        k = C.c_int()
        L.check(L.lib().hdf_batch_get_centers(self._b, int(i), mu.ctypes.data_as(C.c_void_p),
                                              C.byref(k)), "get_centers")
        return mu[: k.value].copy()

    def stats(self, i: int) -> dict:
        s = L.hdf_stats()
        code = L.lib().hdf_batch_get_stats(self._b, int(i), C.byref(s))
        d = {k: getattr(s, k) for k, _ in L.hdf_stats._fields_}
        if code != L.HDF_OK:
            raise L.HDFError(code, f"device status of image {i}")
        return d

    def info(self) -> dict:
        s = L.hdf_batch_info()
        L.check(L.lib().hdf_batch_get_info(self._b, C.byref(s)), "get_info")
        return {k: getattr(s, k) for k, _ in L.hdf_batch_info._fields_}
