"""The phase names of the clustering trace tool cover exactly the phase ids
the clustering kernel records (the TracePhase enum of its argument header)."""
import os
import re

from paper_1811_02363_gb300 import cluster_trace

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_phase_ids_match_the_kernel_enum():
    src = open(os.path.join(ROOT, "paper_1811_02363_gb300", "csrc", "cluster_args.cuh")).read()
    enum = src[src.index("enum TracePhase"):]
    enum = enum[:enum.index("};")]
    ids = {int(v): k[3:] for k, v in re.findall(r"(TR_\w+)\s*=\s*(\d+)", enum)}
    assert ids == cluster_trace.PHASES


def test_timing_tool_names_the_synthetic_workloads():
    from paper_1811_02363_gb300 import synthetic, timing
    for name in timing.WORKLOADS:
        w = synthetic.workload(name)
        assert {"f", "K", "sigma_s", "sigma_r"} <= set(w)


def test_timing_tool_arguments():
    from paper_1811_02363_gb300 import timing
    assert timing.parse_args([]).workloads == timing.WORKLOADS
    a = timing.parse_args(["color2048", "--backward"])
    assert a.workloads == ["color2048"] and a.backward
