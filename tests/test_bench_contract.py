"""The bench line's helpers on the CPU: the algorithmic-byte counts the
roofline divides by, the fields emit() adds to every line, the host record of
the CPU baseline, and the kernel revision that ties a recorded ncu traffic
figure to the source it was measured on."""
import io
import json
import os
import sys
from contextlib import redirect_stdout

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_algorithmic_bytes_of_rmat24():
    # offsets read once, each arc read once, d~ written and read and coreness
    # written once: 8(n+1) + 4 arcs + 12 n
    n, arcs = 1 << 24, 520762754
    assert bench.algorithmic_bytes(n, arcs) == 8 * (n + 1) + 4 * arcs + 12 * n == 2418595344


def test_csr_build_bytes():
    assert bench.csr_build_bytes(10, 7, 12) == 8 * 7 + 8 * 11 + 4 * 12


def test_emit_adds_nominal_fraction_and_host():
    out = {"roofline": {"achieved": 790.0, "unit": "GB/s"}, "cpu_baseline": {"value": 1.0}}
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.emit(out)
    line = json.loads(buf.getvalue())
    assert line["roofline"]["peak_nominal"] == 7900.0
    assert abs(line["roofline"]["frac_nominal"] - 0.1) < 1e-12
    host = line["cpu_baseline"]["host"]
    assert host["logical_cores"] == os.cpu_count() and host["arch"]


def test_emit_leaves_lines_without_roofline_alone():
    buf = io.StringIO()
    with redirect_stdout(buf):
        bench.emit({"impl": "reference", "value": 3.0})
    assert json.loads(buf.getvalue()) == {"impl": "reference", "value": 3.0}


def test_recorded_traffic_is_tied_to_a_kernel_revision():
    # the bench reports the recorded traffic only while kernel_rev equals the
    # hash of the current source, and null after any change to the kernel
    path = os.path.join(ROOT, "profiles", "peel_bsp_rmat24_traffic.json")
    rec = json.load(open(path))
    assert rec["kernel"] == "peel_bsp" and rec["workload"] == "rmat24"
    rev = bench.kernel_revision("peel_bsp.cu")
    assert len(rec["kernel_rev"]) == len(rev) == 12
    # traffic at or above the algorithmic bytes (a copy cannot move less)
    assert rec["dram_bytes_per_launch"] >= bench.algorithmic_bytes(1 << 24, 520762754)


def test_cpu_baseline_protocol_on_a_small_graph():
    """The oracle is timed on the graph it is given, one warm-up then the mean
    of the runs (the paper's protocol, Sec. 6), one host core; the value is
    undirected edges per second of the mean."""
    import graphgen as gg
    import oracle
    n, s, d = gg.disjoint_union((2000, *gg.er(2000, 9000, seed=4)), gg.staircase(30))
    off, adj = oracle.build_csr(n, s, d)
    cb = bench.cpu_oracle_baseline(n, off, adj, "a test graph", warmup=1, runs=3)
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["unit"] == bench.UNIT
    assert cb["s_min"] <= cb["s_mean"]
    assert abs(cb["value"] - (len(adj) // 2) / cb["s_mean"]) <= 1e-6 * cb["value"]
    assert "a test graph" in cb["sample"] and "mean of 3 runs" in cb["sample"]


def test_reference_arm_names_the_gpu_arms_workload():
    """The reference arm decomposes the GPU arm's own graph and names it the
    same way, so both lines describe the same configuration."""
    import inspect
    src = inspect.getsource(bench.run_reference)
    assert "workload_name(args.workload, w)" in src and "make_edges(w)" in src
    assert bench.workload_name("rmat24", bench.WORKLOADS["rmat24"]) == "rmat24: R-MAT scale 24 edge factor 16"


def test_serial_baseline_is_described_as_placed_on_the_timeline():
    assert "not replayed" in bench.SERIAL_NOTE and "arrival timeline" in bench.SERIAL_NOTE
