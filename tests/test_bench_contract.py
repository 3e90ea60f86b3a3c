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
