"""Phase breakdown of the clustering kernel from its device trace.

The clustering launch records, for its block 0, a (phase, time) event at the
end of every step (hdf_get_trace): the distance-statistics passes, the Lloyd
iterations (pass, wait at the grid barrier, reload of the published state),
the partition and the child set-up of every round.  This tool clusters one of
the named synthetic workloads a few times, reads the trace of the last run and
prints the time spent in each phase, its count, and the first events in order.

    python -m paper_1811_02363_gb300.cluster_trace hyper512
"""
from __future__ import annotations

import argparse
import collections
import json

import numpy as np
import torch

from . import api, synthetic

PHASES = {1: "ROOT", 2: "DIST1", 4: "NODE", 5: "LLOYD", 6: "COUNT", 7: "SCATTER", 8: "CHILD",
          9: "LPASS", 11: "LUPDATE", 12: "FWAIT", 13: "FSTAGE", 14: "FDONE", 15: "SETUP",
          16: "DPASS"}


def _median_ms(fn, reps: int = 10) -> float:
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


def breakdown(name: str, first: int = 60) -> dict:
    w = synthetic.workload(name)
    f = torch.from_numpy(w["f"]).cuda()
    n, H, W = f.shape
    if name == "nlm1024":
        flt = api.HDFilter(H, W, n, w["pca_dims"], w["K"], w["sigma_s"], w["sigma_r"])
        p = flt.nlm_guide(f, w["patch"])
    else:
        flt = api.HDFilter(H, W, n, n, w["K"], w["sigma_s"], w["sigma_r"])
        p = f
    try:
        cluster_ms = _median_ms(lambda: flt.cluster(p))
        tr = flt.trace()
        stats = flt.stats()
    finally:
        flt.close()
    total = collections.defaultdict(float)
    count = collections.Counter()
    seq = []
    for i in range(1, len(tr)):
        ph = PHASES.get(int(tr[i, 0]), str(int(tr[i, 0])))
        dt = (tr[i, 1] - tr[i - 1, 1]) / 1e3
        total[ph] += dt
        count[ph] += 1
        if len(seq) < first:
            seq.append((ph, round(float(dt), 1)))
    span = (tr[-1, 1] - tr[0, 1]) / 1e3 if len(tr) else 0.0
    return {"workload": name, "cluster_ms": cluster_ms, "trace_span_us": round(float(span), 1),
            "phases_us": {k: round(v, 1) for k, v in total.items()},
            "phase_counts": dict(count), "first_events_us": seq, "stats": stats}


def main() -> None:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("workload", nargs="?", default="hyper512",
                    choices=["color256", "hyper512", "nlm1024", "color2048"])
    ap.add_argument("--first", type=int, default=60, help="events listed in order")
    args = ap.parse_args()
    print(json.dumps(breakdown(args.workload, args.first)))


if __name__ == "__main__":
    main()
