#!/usr/bin/env python
"""Benchmark of the fast high-dimensional bilateral filter on one or more GPUs.

Workload: hyperspectral bilateral filtering, a 31 x 512 x 512 float32 cube of
smooth spectral mixtures (guide = image), sigma_s = 5 (window 31 x 31),
sigma_r = 0.3, K = 32 centres.  One step = the whole hot path of
Algorithm 1 on the device: bisecting K-means of the guide, the FP64 fit of
A^+, range maps b_k, coefficients c, the K(n+1) spatial convolutions and the
combine/normalise.  Metric: megapixels per second (whole job).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

For N > 1 launch with torchrun (one rank per GPU); every rank filters its
own copy of the workload (replicas, weak scaling) and the slowest rank's time
is used.  ``--impl reference`` times the FP64 CPU oracle (the reference
implementation of this method in this repository) on bounded samples of the
same workload on the host cores.  One JSON line is printed by rank 0.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")   # the CPU oracle runs on one core
os.environ.setdefault("OMP_NUM_THREADS", "1")

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

WORKLOAD = dict(name="hyper512", bands=31, H=512, W=512, sigma_s=5.0, sigma_r=0.3, K=32)
METRIC = "megapixels/s of the fast filter (cluster + fit + filter) on one GB300"
UNIT = "MP/s"
L2_FLUSH_BYTES = 256 << 20          # larger than the 129 MB L2
CPU_SAMPLE = 256                    # crop side of the oracle baseline sample
REF_STEP_CROP = 128                 # crop side of one reference-arm step

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from the
# ncu captures summarised under profiles/, valid only for the kernel source they
# were taken on (sha256 prefix of the file that holds the kernel).
NCU_TRAFFIC = {
    "cluster_kernel": ("paper_1811_02363_gb300/csrc/cluster_kernel.cuh", "c017618119d5", 202.75e6),
    "filter_tile_kernel": ("paper_1811_02363_gb300/csrc/filter_tile.cuh", "eacdca9e8b1b", 247.96e6),
}


def ncu_traffic(kernel: str):
    import hashlib
    path, sha, nbytes = NCU_TRAFFIC[kernel]
    try:
        cur = hashlib.sha256(open(os.path.join(ROOT, path), "rb").read()).hexdigest()[:12]
    except OSError:
        return None
    return nbytes if cur == sha else None


def config(extra=None):
    c = {"workload": "hyperspectral bilateral 31x512x512, sigma_s=5 (31x31 window), "
                     "sigma_r=0.3, K=32, guide=image",
         "pixels_per_step": WORKLOAD["H"] * WORKLOAD["W"], "channels": 31, "K": 32, "S": 15,
         "l2": "flushed between timed steps (256 MB write)"}
    if extra:
        c.update(extra)
    return c


def slowest_rank_ms(ms: float, dist, device) -> float:
    """The job's time: the maximum over ranks of a rank's timed region (ms)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_mps(units_per_rank: int, world: int, steps: int, ms: float) -> float:
    """Whole-job megapixels per second: every rank filters its own replica
    (weak scaling), so the job's pixels are world * steps * units_per_rank."""
    return world * steps * units_per_rank / (ms * 1e-3) / 1e6


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


# ---------------------------------------------------------------- CPU oracle

def oracle_mps(crop: int) -> tuple[float, float]:
    """Time the FP64 oracle (bisecting K-means + Algorithm 1) on a crop of the
    workload; returns (MP/s, seconds)."""
    from oracle import hdfilter_oracle as O
    from paper_1811_02363_gb300 import synthetic
    f = synthetic.hyperspectral_mixture(WORKLOAD["H"], WORKLOAD["W"], bands=31, seed=1)
    f = f[:, :crop, :crop].astype(np.float64)
    t0 = time.perf_counter()
    mu, _, _ = O.bisecting_kmeans(f.reshape(31, -1).T, WORKLOAD["K"])
    O.fast_filter(f, f, mu, WORKLOAD["sigma_s"], WORKLOAD["sigma_r"], 15)
    dt = time.perf_counter() - t0
    return crop * crop / dt / 1e6, dt


def run_reference(args) -> None:
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_mps(REF_STEP_CROP)
    times = []
    for _ in range(args.steps):
        _, dt = oracle_mps(REF_STEP_CROP)
        times.append(dt)
    total = sum(times)
    value = args.steps * REF_STEP_CROP ** 2 / total / 1e6
    sample = f"{REF_STEP_CROP}x{REF_STEP_CROP} crop of the workload per step (all 31 bands, K=32)"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config({"reference": "FP64 CPU oracle (numpy), 1 host core"}),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU

class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines, self.n0 = [], 0

    def start(self):
        """Start sampling every 50 ms and return once the first sample is in, so
        that the samples cover the timed region that follows."""
        import threading
        self.lines = []
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        first = threading.Event()

        def reader():
            for line in self.proc.stdout:
                self.lines.append(line)
                first.set()
            first.set()

        self.thread = threading.Thread(target=reader, daemon=True)
        self.thread.start()
        first.wait(timeout=10.0)
        self.n0 = len(self.lines)   # samples taken before the timed region

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            self.proc.wait()
        self.thread.join(timeout=5)
        return self.summarize(self.lines[self.n0:] or self.lines)

    @staticmethod
    def summarize(lines) -> dict:
        """Median SM clock, maximum clock and the throttle reasons seen, from
        nvidia-smi CSV lines (no header, no units) of FIELDS."""
        out = "".join(lines)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def run_gpu(args) -> None:
    import torch
    from paper_1811_02363_gb300 import api, synthetic

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    H, W, K = WORKLOAD["H"], WORKLOAD["W"], WORKLOAD["K"]
    f_host = synthetic.hyperspectral_mixture(H, W, bands=31, seed=1)
    f = torch.from_numpy(f_host).to(dev)
    g = torch.empty_like(f)
    flt = api.HDFilter(H, W, 31, 31, K, WORKLOAD["sigma_s"], WORKLOAD["sigma_r"])
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        flt.cluster(f)
        flt.apply(f, f, g)

    args.warmup = max(args.warmup, 3)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if args.stage != "all":
        # profiling aid: run one stage --steps times and stop (no JSON line)
        for _ in range(args.steps):
            if args.stage == "cluster":
                flt.cluster(f)
            else:
                flt.apply(f, f, g)
        torch.cuda.synchronize()
        print(f"stage {args.stage} x{args.steps} done; stats {flt.stats()}", flush=True)
        return

    # ---- device-resident timing, one event pair per step, L2 flushed outside
    clocks = ClockSampler(local)
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    # dominant-kernel timing: the same steps split at the cluster/filter boundary
    mid = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    for i in range(args.steps):
        flush.zero_()
        ev[i][0].record(stream)
        flt.cluster(f)
        mid[i].record(stream)
        flt.apply(f, f, g)
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    cluster_ms = [a.elapsed_time(m) for (a, _), m in zip(ev, mid)]
    apply_ms = [m.elapsed_time(b) for (_, b), m in zip(ev, mid)]
    total_ms = slowest_rank_ms(sum(step_ms), dist, dev)
    value = job_mps(H * W, ws, args.steps, total_ms)

    # ---- filter-kernel timing (CUDA events around apply only, same stream)
    ta = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    for i in range(args.steps):
        flush.zero_()
        ta[i][0].record(stream)
        flt.apply(f, f, g)
        ta[i][1].record(stream)
    torch.cuda.synchronize()
    apply_only_ms = statistics.median(a.elapsed_time(b) for a, b in ta)

    # ---- end to end through the C ABI with host buffers: every step copies its
    # image from pinned host memory and reads its result back; the copies run on
    # a copy stream, double-buffered, overlapping the neighbouring steps' compute
    # (step i + 1's upload and step i's read-back run while the GPU filters).
    f_pin = torch.from_numpy(f_host).pin_memory()
    g_pin = torch.empty_like(f_pin).pin_memory()
    f_e = [torch.empty_like(f) for _ in range(2)]
    g_e = [torch.empty_like(f) for _ in range(2)]
    copy = torch.cuda.Stream(device=dev)
    up = [torch.cuda.Event() for _ in range(2)]      # upload into f_e[b] done
    done = [torch.cuda.Event() for _ in range(2)]    # step on buffer b computed
    back = [torch.cuda.Event() for _ in range(2)]    # g_e[b] read back
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    e0.record(stream)
    copy.wait_stream(stream)

    def upload(b):
        with torch.cuda.stream(copy):
            f_e[b].copy_(f_pin, non_blocking=True)
            up[b].record(copy)

    upload(0)
    for i in range(args.steps):
        b = i & 1
        if i + 1 < args.steps:
            if i >= 1:
                copy.wait_event(done[b ^ 1])   # step i - 1 no longer reads f_e[b ^ 1]
            upload(b ^ 1)
        stream.wait_event(up[b])
        if i >= 2:
            stream.wait_event(back[b])         # step i - 2's result has left g_e[b]
        flt.cluster(f_e[b])
        flt.apply(f_e[b], f_e[b], g_e[b])
        done[b].record(stream)
        with torch.cuda.stream(copy):
            copy.wait_event(done[b])
            g_pin.copy_(g_e[b], non_blocking=True)
            back[b].record(copy)
    stream.wait_stream(copy)
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_same = bool(torch.equal(g_pin, g.cpu()))   # the read-back equals the resident run
    g = g_e[(args.steps - 1) & 1]
    e2e_ms = slowest_rank_ms(e0.elapsed_time(e1), dist, dev)
    e2e_value = job_mps(H * W, ws, args.steps, e2e_ms)
    nbytes = f_host.nbytes

    # ---- brute force on the same GPU (Eq. (1)-(2)) and the accuracy of the fast filter
    gb = api.bruteforce(f, None, WORKLOAD["sigma_s"], WORKLOAD["sigma_r"])
    torch.cuda.synchronize()
    b0, b1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    b0.record(stream)
    api.bruteforce(f, None, WORKLOAD["sigma_s"], WORKLOAD["sigma_r"], out=gb)
    b1.record(stream)
    torch.cuda.synchronize()
    brute_ms = b0.elapsed_time(b1)
    flt.cluster(f)
    flt.apply(f, f, g)
    mse = float(torch.mean((g.double() - gb.double()) ** 2).item())
    psnr = float("inf") if mse == 0 else -10.0 * np.log10(mse)
    # band-averaged PSNR (MPSNR, the hyperspectral quality figure of Sec. IV)
    band_mse = torch.mean((g.double() - gb.double()) ** 2, dim=(1, 2)).cpu().numpy()
    mpsnr = float(np.mean([float("inf") if m == 0 else -10.0 * np.log10(m) for m in band_mse]))
    st = flt.stats()

    # ---- the box spatial kernel (omega = 1 on W, Sec. III's NLM kernel) on the
    # same image and centres: apply-only time and PSNR against its brute force
    fb = api.HDFilter(H, W, 31, 31, K, WORKLOAD["sigma_s"], WORKLOAD["sigma_r"], S=15, spatial="box")
    fb.set_centers(flt.get_centers())
    gbx = torch.empty_like(f)
    fb.apply(f, f, gbx)
    tb = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    for i in range(args.steps):
        flush.zero_()
        tb[i][0].record(stream)
        fb.apply(f, f, gbx)
        tb[i][1].record(stream)
    torch.cuda.synchronize()
    box_ms = statistics.median(a.elapsed_time(b) for a, b in tb)
    gbb = api.bruteforce(f, None, WORKLOAD["sigma_s"], WORKLOAD["sigma_r"], S=15, spatial="box")
    torch.cuda.synchronize()
    bmse = float(torch.mean((gbx.double() - gbb.double()) ** 2).item())
    box = {"spatial": "box, S=15 (31x31 window), same centres", "apply_ms": box_ms,
           "apply_mps": H * W / (box_ms * 1e-3) / 1e6,
           "psnr_vs_box_bruteforce_db": float("inf") if bmse == 0 else -10.0 * np.log10(bmse)}
    fb.close()

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    # ---- roofline of the dominant kernel and of the filter kernel
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    sm_max = peaks.get("sm_max_mhz", 2070.0)
    fp32_peak_tflops = 152 * 128 * 2 * sm_max * 1e6 / 1e12
    npx = H * W
    # Clustering: a model of plain Lloyd traffic, rho*4 B per point
    # per assignment pass, 20 passes per level, log2 K levels.
    cl_bytes = npx * 31 * 4 * 20 * 5
    cl_s = statistics.median(cluster_ms) * 1e-3
    # Filter: 4 (2S+1) K (n+1) FLOP per pixel for the two 1-D passes (FMA = 2).
    fir_flops = npx * 4 * (2 * 15 + 1) * K * 32
    ap_s = apply_only_ms * 1e-3
    rf_cluster = {"kernel": "cluster_kernel", "bound": "hbm", "achieved": cl_bytes / cl_s / 1e9,
                  "peak": hbm, "unit": "GB/s", "frac": cl_bytes / cl_s / 1e9 / hbm,
                  "traffic": ncu_traffic("cluster_kernel"), "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)",
                  "algorithmic_bytes_per_launch": cl_bytes}
    rf_filter = {"kernel": "filter_tile_kernel (+ range maps, divide)", "bound": "alu",
                 "achieved": fir_flops / ap_s / 1e12, "peak": fp32_peak_tflops,
                 "unit": "TFLOP/s", "frac": fir_flops / ap_s / 1e12 / fp32_peak_tflops,
                 "traffic": ncu_traffic("filter_tile_kernel"),
                 "peak_source": "152 SM x 128 FP32 lanes x 2 x max SM clock (derived)",
                 "algorithmic_flops_per_launch": fir_flops}
    dominant = rf_cluster if statistics.median(cluster_ms) >= apply_only_ms else rf_filter

    cpu = None
    if ws == 1 or rank == 0:
        cpu_v, cpu_s = oracle_mps(CPU_SAMPLE)
        cpu = {"value": cpu_v, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{CPU_SAMPLE}x{CPU_SAMPLE} crop of the workload, clustering + "
                         f"Algorithm 1 in FP64 ({cpu_s:.1f} s)"}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": config({"parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"}),
            "roofline": dominant,
            "roofline_kernels": [rf_cluster, rf_filter],
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": nbytes,
                    "d2h_bytes_per_step": nbytes,
                    "copies": "pinned, on a copy stream, double-buffered, overlapping the "
                              "neighbouring steps' compute",
                    "result_equals_resident_run": e2e_same},
            "gpu_launches": 6 * args.steps,
            "clocks": clk,
            "breakdown_ms": {"cluster_fit": statistics.median(cluster_ms),
                             "apply": statistics.median(apply_ms),
                             "apply_only": apply_only_ms},
            "bruteforce_gpu": {"value": npx / (brute_ms * 1e-3) / 1e6, "unit": UNIT,
                               "ms": brute_ms},
            "psnr_vs_bruteforce_db": psnr,
            "mpsnr_vs_bruteforce_db": mpsnr,
            "box_kernel": box,
            "stats": st}
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--stage", default="all", choices=["all", "apply", "cluster"],
                    help="profiling aid: run only this stage after the warm-up")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
