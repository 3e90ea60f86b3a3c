"""Benchmark of the GB300 k-core peel (one JSON line on rank 0).

Default workload: R-MAT scale 24, edge factor 16, (a,b,c,d) = (.57,.19,.19,.05),
ids permuted, symmetrised and deduplicated (the paper's power-law class,
Sec. 6.1). A step is one full decomposition (kcore_decompose: degree init,
frontier extraction, peel, next-level search, all levels) of the graph held in
HBM; the CSR build from the raw edge list is timed once beside it. The metric
is undirected edges per second (each edge counted once per decomposition).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                    [--workload rmat24|rmat22|er10k]

Multi-GPU: a single graph does not shard (each level depends on all earlier
decrements), so N ranks run N independent replicas ("replicas only") and
`value` sums their throughput; the timed region is bracketed by a barrier and
the slowest rank's time is used.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "k-core edges/s (GTEPS) & % HBM roofline; batched graphs/s + p99 vs plain loop"
UNIT = "undirected edges/s"
L2_BYTES = 129 * 1024 * 1024


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


WORKLOADS = {
    "rmat24": dict(kind="rmat", scale=24, ef=16),
    "rmat22": dict(kind="rmat", scale=22, ef=16),
    "er10k": dict(kind="er", n=10_000, m=50_000),
}


def make_edges(w):
    import graphgen as gg
    if w["kind"] == "rmat":
        n = 1 << w["scale"]
        s, d = gg.rmat(w["scale"], w["ef"], seed=1, perm_seed=2)
        return n, s, d
    n = w["n"]
    s, d = gg.er(n, w["m"], seed=1)
    return n, s, d


def algorithmic_bytes(n: int, arcs: int) -> int:
    """Minimum traffic of one decomposition: offsets read once (8(n+1)), each
    adjacency list read once (4 * arcs), induced degrees written once and read
    once plus coreness written once (12 n)."""
    return 8 * (n + 1) + 4 * arcs + 12 * n


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(self.index)], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (FileNotFoundError, OSError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_oracle_baseline(scale: int = 22, reps: int = 1):
    """The oracle (sequential Batagelj-Zaversnik in C, one host core) on an
    R-MAT graph of the same generator and parameters at a smaller scale."""
    import graphgen as gg
    import oracle
    s, d = gg.rmat(scale, 16, seed=1, perm_seed=2)
    n = 1 << scale
    off, adj = oracle.build_csr(n, s, d)
    ts = []
    for _ in range(reps):
        t0 = time.perf_counter()
        oracle.bz(n, off, adj)
        ts.append(time.perf_counter() - t0)
    t = min(ts)
    return {"value": (len(adj) // 2) / t, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"Batagelj-Zaversnik on R-MAT scale {scale} (same generator, edge factor 16; "
                      f"{len(adj) // 2} undirected edges), best of {reps}, {t:.2f} s"}


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    import graphgen as gg
    import oracle
    scale = 20
    s, d = gg.rmat(scale, 16, seed=1, perm_seed=2)
    n = 1 << scale
    off, adj = oracle.build_csr(n, s, d)
    mu = len(adj) // 2
    for _ in range(args.warmup):
        oracle.bz(n, off, adj)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.bz(n, off, adj)
    dt = time.perf_counter() - t0
    value = mu * args.steps / dt
    sample = (f"each step: Batagelj-Zaversnik on R-MAT scale {scale} (same generator as "
              f"{args.workload}, {mu} undirected edges), 1 host core")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": f"{args.workload} (CPU sample: rmat{scale})", "parallelism": "none"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_gpu(args):
    import torch
    import torch.distributed as dist

    from paper_2502_08042_gb300 import KCore

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = WORKLOADS[args.workload]
    n, s, d = make_edges(w)
    E = len(s)
    k = KCore(local)
    S = torch.from_numpy(s).to(dev)
    D = torch.from_numpy(d).to(dev)
    del s, d
    # ---- CSR build (a1), timed separately
    csr_ms = []
    for i in range(3):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record()
        off, adj_buf, m_t = k.build_csr(n, S, D, sync=False)
        ev1.record()
        k.sync()
        csr_ms.append(ev0.elapsed_time(ev1))
    m = int(m_t.item())
    adj = adj_buf[:m].clone()
    del adj_buf, S, D
    torch.cuda.empty_cache()
    mu = m // 2
    core = torch.empty(n, dtype=torch.int32, device=dev)
    kmax = torch.empty(1, dtype=torch.int32, device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        k.decompose(off, adj, core, kmax, sync=False)

    for _ in range(args.warmup):
        step()
        k.sync()
    st = k.stats()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        for i in range(args.steps):
            flush.zero_()  # write a buffer larger than L2 between timed steps
            evs[i][0].record(stream)
            step()
            evs[i][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    k.sync()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = sum(step_ms)
    if ws > 1:
        t = torch.tensor([total_ms], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    value = ws * mu * args.steps / (total_ms / 1e3)

    # ---- end to end through the C ABI with host buffers
    off_h = torch.empty(n + 1, dtype=torch.int64, pin_memory=True)
    adj_h = torch.empty(m, dtype=torch.int32, pin_memory=True)
    off_h.copy_(off)
    adj_h.copy_(adj)
    core_h = torch.empty(n, dtype=torch.int32, pin_memory=True)
    km_h = torch.empty(1, dtype=torch.int32, pin_memory=True)
    on, an, cn, kn = off_h.numpy(), adj_h.numpy(), core_h.numpy(), km_h.numpy()
    for _ in range(2):
        k.decompose_host_into(on, an, cn, kn)
    e2e_steps = max(2, min(args.steps, 5))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        k.decompose_host_into(on, an, cn, kn)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e = {"value": ws * mu / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 8 * (n + 1) + 4 * m,
           "d2h_bytes_per_step": 4 * n + 4, "ms_per_step": e2e_s * 1e3}

    if rank != 0:
        if ws > 1:
            dist.barrier()
        return
    peak, peak_kind = load_peaks()
    bmin = algorithmic_bytes(n, m)
    achieved = bmin / (ms_per_step / 1e3) / 1e9
    traffic = None
    tp = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tp):
        with open(tp) as f:
            tj = json.load(f)
        if tj.get("workload") == args.workload and tj.get("kernel_rev") == kernel_revision():
            traffic = tj.get("dram_bytes_per_launch")
    cpu = None
    if not args.no_cpu_baseline:
        cpu = cpu_oracle_baseline()
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {
            "workload": f"{args.workload}: R-MAT scale {w.get('scale')} edge factor {w.get('ef')}"
            if w["kind"] == "rmat" else f"{args.workload}: Erdos-Renyi n={w['n']} m={w['m']}",
            "n": n, "edges_drawn": E, "undirected_edges": mu, "arcs": m, "kmax": int(kmax.item()),
            "rounds": st["rounds"], "empty_rounds": st["empty_rounds"], "grid": st["grid"],
            "l2": "inputs larger than L2 and a 258 MB buffer written between timed steps",
            "csr_build_ms": min(csr_ms), "parallelism": "replicas" if ws > 1 else "single GPU",
            "wall_s": wall,
        },
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                     "algorithmic_bytes": bmin, "kernel": "peel_persistent"},
        "e2e": e2e,
        "gpu_launches": args.steps,
        "cpu_baseline": cpu,
    }
    clocks = clk.summary()
    if clocks:
        out["clocks"] = clocks
    print(json.dumps(out), flush=True)
    if ws > 1:
        dist.barrier()


def kernel_revision() -> str:
    """Hash of the peel kernel source, to tie recorded ncu traffic to it."""
    import hashlib
    p = os.path.join(ROOT, "paper_2502_08042_gb300", "csrc", "peel.cu")
    with open(p, "rb") as f:
        return hashlib.sha1(f.read()).hexdigest()[:12]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="rmat24", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
