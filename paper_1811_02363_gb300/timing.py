"""Stage timings of the named synthetic workloads on the current GPU.

For each workload: the PCA guide (nonlocal means), the clustering, the filter
apply with the Gaussian, box and recursive-Gaussian spatial kernels, with
--bruteforce the brute force of Eq. (1)-(2), and with --backward the gradient
pass (dL/df, dL/dlog sigma_s, dL/dlog sigma_r) of the Gaussian filter for a
random upstream gradient, on its own and right after the forward pass (whose
state it then reuses).  Times are medians of CUDA
events on the current stream, inputs resident on the device.

    python -m paper_1811_02363_gb300.timing hyper512 color2048 --backward --bruteforce
"""
from __future__ import annotations

import argparse
import json
import math

import numpy as np
import torch

from . import api, synthetic

WORKLOADS = ["color256", "hyper512", "nlm1024", "color2048"]


def median_ms(fn, reps: int = 10) -> float:
    s = torch.cuda.current_stream()
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        fn()
        b.record(s)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return float(np.median(ts))


def median_ms_after(pre, fn, reps: int = 10) -> float:
    """Median ms of fn alone, each run preceded by an untimed pre()."""
    s = torch.cuda.current_stream()
    pre()
    fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        pre()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(s)
        fn()
        b.record(s)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return float(np.median(ts))


def workload_times(name: str, backward: bool = False, bruteforce: bool = False) -> dict:
    w = synthetic.workload(name)
    f = torch.from_numpy(w["f"]).cuda()
    n, H, W = f.shape
    nlm = name == "nlm1024"
    rho = w["pca_dims"] if nlm else n
    out = {"workload": name, "pixels": H * W, "K": w["K"], "sigma_s": w["sigma_s"],
           "sigma_r": w["sigma_r"]}
    g = torch.empty_like(f)
    centres = None
    for spatial in ("gauss", "box", "young"):
        flt = api.HDFilter(H, W, n, rho, w["K"], w["sigma_s"], w["sigma_r"], spatial=spatial)
        try:
            p = flt.nlm_guide(f, w["patch"]) if nlm else f
            if spatial == "gauss":
                if nlm:
                    out["guide_ms"] = median_ms(lambda: flt.nlm_guide(f, w["patch"], out=p))
                out["S"] = int(math.ceil(3.0 * w["sigma_s"]))
                out["cluster_ms"] = median_ms(lambda: flt.cluster(p))
                centres = flt.get_centers()
            else:
                flt.set_centers(centres)
            out[f"apply_{spatial}_ms"] = median_ms(lambda: flt.apply(f, p, g))
            if backward and spatial == "gauss":
                G = torch.randn(f.shape, device=f.device, dtype=f.dtype,
                                generator=torch.Generator(device=f.device).manual_seed(5))
                out["backward_ms"] = median_ms(lambda: flt.backward(f, p, G))
                # right after the forward pass: its state reused (hdf_backward_after_apply)
                out["backward_after_apply_ms"] = median_ms_after(
                    lambda: flt.apply(f, p, g), lambda: flt.backward(f, p, G, g=g))
            out[f"stats_{spatial}"] = flt.stats()
            if bruteforce and spatial == "gauss":   # Eq. (1)-(2) on the same guide
                gb = api.bruteforce(f, p, w["sigma_s"], w["sigma_r"])
                out["bruteforce_ms"] = median_ms(
                    lambda: api.bruteforce(f, p, w["sigma_s"], w["sigma_r"], out=gb), reps=3)
        finally:
            flt.close()
    return out


def parse_args(argv=None) -> argparse.Namespace:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("workloads", nargs="*", metavar="workload",
                    help=f"one or more of {', '.join(WORKLOADS)} (default: all)")
    ap.add_argument("--backward", action="store_true", help="also time the gradient pass")
    ap.add_argument("--bruteforce", action="store_true",
                    help="also time the brute-force filter (Eq. (1)-(2))")
    args = ap.parse_args(argv)
    bad = [w for w in args.workloads if w not in WORKLOADS]
    if bad:
        ap.error(f"unknown workload(s) {bad}; choose from {WORKLOADS}")
    args.workloads = args.workloads or list(WORKLOADS)
    return args


def main() -> None:
    args = parse_args()
    for name in args.workloads:
        print(json.dumps(workload_times(name, args.backward, args.bruteforce)), flush=True)


if __name__ == "__main__":
    main()
