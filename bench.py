"""Benchmark of the GB300 k-core peel (one JSON line on rank 0).

Default workload: R-MAT scale 24, edge factor 16, (a,b,c,d) = (.57,.19,.19,.05),
ids permuted, symmetrised and deduplicated (the paper's power-law class,
Sec. 6.1). A step is one full decomposition (kcore_decompose: degree init,
frontier extraction, peel, next-level search, all levels) of the graph held in
HBM; the CSR build from the raw edge list is timed once beside it. The metric
is undirected edges per second (each edge counted once per decomposition).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                    [--workload rmat24|rmat22|er10k|knn|batched|served|kquery]

Other workloads (one JSON line each): `knn` is the 10-NN graph of 2^24 uniform
points plus 64 planted cliques; `batched` decomposes the 4,096-graph batch in
one launch (graphs/s, against a loop of single-graph launches on the same
graphs with identical output); `served` streams 2,000 requests (95% drawn from
the batch distribution, 5% R-MAT scale 20..24) at Poisson arrival rates and
reports p50/p99 latency and graphs/s against serial plain launches.

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


NOMINAL_PEAK = {"GB/s": 7900.0, "TFLOP/s": 2250.0}  # GB300 datasheet: HBM3e, dense bf16


def host_cpu() -> dict:
    """Model, architecture and logical cores of the host the CPU legs ran on."""
    import platform
    model = None
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                key = line.split(":")[0].strip().lower()
                if key in ("model name", "hardware", "cpu model"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    if not model:
        # Arm hosts name the core in lscpu's "Model name" rather than /proc/cpuinfo
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=5).stdout
            for line in out.splitlines():
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except (OSError, subprocess.SubprocessError):
            pass
    return {"model": model or platform.processor() or None, "arch": platform.machine(),
            "logical_cores": os.cpu_count()}


def emit(out: dict) -> None:
    """Prints the bench line, adding the roofline fraction of the nominal peak
    beside the measured one and the host CPU beside the CPU baseline."""
    rf = out.get("roofline")
    if rf and rf.get("achieved") is not None and rf.get("unit") in NOMINAL_PEAK:
        rf["peak_nominal"] = NOMINAL_PEAK[rf["unit"]]
        rf["frac_nominal"] = rf["achieved"] / NOMINAL_PEAK[rf["unit"]]
    cb = out.get("cpu_baseline")
    if cb:
        cb["host"] = host_cpu()
    print(json.dumps(out), flush=True)


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
    "knn": dict(kind="knn", n=1 << 24, k=10, cliques=64),
    "batched": dict(kind="batched", G=4096),
    "served": dict(kind="served", requests=2000),
    "kquery": dict(kind="kquery", scale=24, ef=16, kprimes=(16, 128, 1024)),
}


def make_edges(w):
    import graphgen as gg
    if w["kind"] == "rmat":
        n = 1 << w["scale"]
        s, d = gg.rmat(w["scale"], w["ef"], seed=1, perm_seed=2)
        return n, s, d
    if w["kind"] == "knn":
        n, s, d, sizes, members = gg.workload_knn_cliques(w["n"], w["k"], w["cliques"])
        return n, s, d
    n = w["n"]
    s, d = gg.er(n, w["m"], seed=1)
    return n, s, d


def workload_name(name, w):
    if w["kind"] == "rmat":
        return f"{name}: R-MAT scale {w['scale']} edge factor {w['ef']}"
    if w["kind"] == "knn":
        return f"{name}: 10-NN of 2^24 uniform points + 64 planted cliques (sizes 50..2000)"
    return f"{name}: Erdos-Renyi n={w['n']} m={w['m']}"


def csr_build_bytes(n: int, edges: int, arcs: int) -> int:
    """Minimum traffic of one CSR build: the edge list read once (8 bytes per
    pair), offsets and adjacency written once."""
    return 8 * edges + 8 * (n + 1) + 4 * arcs


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


def max_over_ranks(x: float, ws: int, device=None) -> float:
    """The slowest rank's value, which is the job's time: an all-reduce MAX over
    the process group (a device tensor with NCCL, a host tensor with gloo)."""
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = device if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, ws: int, max_ms: float) -> float:
    """Weak scaling, replicas: every rank decomposes its own copy, so the job
    processed ws x units in the slowest rank's time."""
    return ws * units_per_rank / (max_ms / 1e3)


def cpu_oracle_baseline(n: int, off, adj, what: str, warmup: int = 1, runs: int = 5):
    """The oracle (sequential Batagelj-Zaversnik in C, one host core) on the
    very CSR the GPU decomposes, with the paper's protocol (Sec. 6: one
    warm-up, then the mean of five runs; the minimum is reported beside it)."""
    import oracle
    for _ in range(warmup):
        oracle.bz(n, off, adj)
    ts = []
    for _ in range(runs):
        t0 = time.perf_counter()
        oracle.bz(n, off, adj)
        ts.append(time.perf_counter() - t0)
    mean, best = sum(ts) / len(ts), min(ts)
    mu = len(adj) // 2
    return {"value": mu / mean, "unit": UNIT, "cores": 1, "kind": "oracle",
            "value_min_time": mu / best, "s_mean": mean, "s_min": best,
            "sample": f"Batagelj-Zaversnik on the bench's own graph ({what}, {mu} undirected edges), "
                      f"{warmup} warm-up + mean of {runs} runs ({mean:.2f} s mean, {best:.2f} s min), "
                      f"one host core"}


def run_kquery(args):
    """The k'-core query (App. B) on R-MAT scale 24 at thresholds 16, 128 and
    1024 (the paper's range is 16..2048), beside the full decomposition of the
    same graph; value = undirected edges per second at the middle threshold."""
    import torch

    import graphgen as gg
    from paper_2502_08042_gb300 import KCore

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = WORKLOADS["kquery"]
    n = 1 << w["scale"]
    s, d = gg.rmat(w["scale"], w["ef"], seed=1, perm_seed=2)
    k = KCore(local)
    off, adj_buf, m_t = k.build_csr(n, torch.from_numpy(s).to(dev), torch.from_numpy(d).to(dev), sync=False)
    k.sync()
    del s, d
    m = int(m_t.item())
    adj = adj_buf[:m].clone()
    del adj_buf
    torch.cuda.empty_cache()
    mu = m // 2
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device=dev)
    mask = torch.empty(n, dtype=torch.int32, device=dev)
    size = torch.empty(1, dtype=torch.int64, device=dev)
    core = torch.empty(n, dtype=torch.int32, device=dev)
    kmax = torch.empty(1, dtype=torch.int32, device=dev)

    def timed(fn):
        for _ in range(args.warmup):
            fn()
            k.sync()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        torch.cuda.synchronize()
        for i in range(args.steps):
            flush.zero_()
            evs[i][0].record()
            fn()
            evs[i][1].record()
        torch.cuda.synchronize()
        k.sync()
        return sum(a.elapsed_time(b) for a, b in evs) / args.steps

    with ClockSampler(local) as clk:
        full_ms = timed(lambda: k.decompose(off, adj, core, kmax, sync=False))
        per = []
        for kp in w["kprimes"]:
            ms = timed(lambda: k.core_mask(off, adj, kp, mask, size, sync=False))
            st = k.stats()
            c = core.cpu().numpy()
            same = bool((mask.cpu().numpy() == (c >= kp)).all())
            per.append({"kprime": kp, "ms": ms, "core_size": int(size.item()), "passes": st["passes"],
                        "matches_coreness_ge_kprime": same, "edges_per_s": mu / (ms / 1e3)})
    mid = per[len(per) // 2]
    cpu = None
    if not args.no_cpu_baseline:
        import oracle
        ss, dd = gg.rmat(22, 16, seed=1, perm_seed=2)
        o2, a2 = oracle.build_csr(1 << 22, ss, dd)
        t0 = time.perf_counter()
        oracle.kcore_mask(1 << 22, o2, a2, mid["kprime"])
        t = time.perf_counter() - t0
        cpu = {"value": (len(a2) // 2) / t, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"repeated deletion (k'={mid['kprime']}) on R-MAT scale 22, {len(a2) // 2} "
                         f"undirected edges, {t:.2f} s"}
    peak, peak_kind = load_peaks()
    bmin = 8 * (n + 1) + 4 * m + 8 * n  # offsets, lists once, d~ written and read, mask written
    out = {
        "metric": METRIC, "value": mid["edges_per_s"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": mid["ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": f"kquery: k'-core of R-MAT scale {w['scale']} edge factor {w['ef']}",
                   "n": n, "arcs": m, "kprime": mid["kprime"], "per_kprime": per,
                   "full_decomposition_ms": full_ms,
                   "l2": "inputs larger than L2 and a 258 MB buffer written between timed steps"},
        "roofline": {"bound": "hbm", "achieved": bmin / (mid["ms"] / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": bmin / (mid["ms"] / 1e3) / 1e9 / peak, "traffic": None, "peak_kind": peak_kind,
                     "algorithmic_bytes": bmin, "kernel": "peel_bsp"},
        "e2e": None, "gpu_launches": args.steps, "cpu_baseline": cpu,
    }
    cl = clk.summary()
    if cl:
        out["clocks"] = cl
    emit(out)


def run_reference(args):
    """The oracle on the GPU arm's own workload: each step is one
    Batagelj-Zaversnik decomposition (one host core) of the same graph, from
    the same generator, built by the oracle's CSR builder (not timed)."""
    ws, rank, local = dist_env()
    if rank != 0:
        return
    import oracle
    w = WORKLOADS[args.workload]
    if w["kind"] not in ("rmat", "knn", "er"):
        emit({"impl": "reference", "unavailable": f"no CPU reference arm for the {args.workload} workload"})
        return
    n, s, d = make_edges(w)
    E = len(s)
    off, adj = oracle.build_csr(n, s, d)
    del s, d
    mu = len(adj) // 2
    for _ in range(args.warmup):
        oracle.bz(n, off, adj)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.bz(n, off, adj)
    dt = time.perf_counter() - t0
    value = mu * args.steps / dt
    sample = (f"each step: Batagelj-Zaversnik on the whole {workload_name(args.workload, w)} graph "
              f"({mu} undirected edges), 1 host core")
    emit({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": workload_name(args.workload, w), "n": n, "edges_drawn": E,
                   "undirected_edges": mu, "arcs": len(adj), "parallelism": "none"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    })


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
    variant = {}
    if args.sampling:
        variant.update(sampling=1, sample_mu=args.sample_mu, sample_threshold=args.sample_threshold,
                       sample_check=0 if args.no_sample_check else 1)
    if args.warp_combine:
        variant.update(warp_combine=1)
    k = KCore(local, sync_mode=args.sync_mode, **variant)
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
    total_ms = max_over_ranks(sum(step_ms), ws, dev)
    ms_per_step = total_ms / args.steps
    value = job_throughput(mu * args.steps, ws, total_ms)

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
    e2e_s = max_over_ranks((time.perf_counter() - t0) / e2e_steps * 1e3, ws, dev) / 1e3
    e2e = {"value": job_throughput(mu, ws, e2e_s * 1e3), "unit": UNIT, "h2d_bytes_per_step": 8 * (n + 1) + 4 * m,
           "d2h_bytes_per_step": 4 * n + 4, "ms_per_step": e2e_s * 1e3}

    if rank != 0:
        if ws > 1:
            dist.barrier()
        return
    peak, peak_kind = load_peaks()
    bmin = algorithmic_bytes(n, m)
    achieved = bmin / (ms_per_step / 1e3) / 1e9
    kname, ksrc = PEEL_KERNELS[st["sync_mode"]]
    traffic = None
    # recorded traffic belongs to the default schedule of its kernel
    tp = os.path.join(ROOT, "profiles", f"{kname}_{args.workload}_traffic.json")
    if st["sync_mode"] == 3 or variant:
        tp = ""
    if os.path.exists(tp):
        with open(tp) as f:
            tj = json.load(f)
        if tj.get("workload") == args.workload and tj.get("kernel_rev") == kernel_revision(ksrc):
            traffic = tj.get("dram_bytes_per_launch")
    # the synchronisation floor: grid barriers taken x the measured latency of
    # one barrier on the same grid (tail phases end at a CTA barrier instead)
    bar_ns = k.barrier_latency_ns(grid=st["grid"], iters=2000)
    sync_floor = {"barriers": st["barriers"], "barrier_us": bar_ns / 1e3,
                  "ms": st["barriers"] * bar_ns / 1e6, "tail_phases": st["tail_phases"]}
    cpu = None
    if not args.no_cpu_baseline:
        cpu = cpu_oracle_baseline(n, off.cpu().numpy(), adj.cpu().numpy(), workload_name(args.workload, w))
    kmax_val = int(kmax.item())
    # the batched form of the same peel, measured in the same run (one GPU):
    # graphs/s against a loop of plain launches, with identical output
    batched = None
    if args.workload == "rmat24" and ws == 1 and not args.no_batched:
        del off, adj, core, kmax, flush, adj_h, off_h, core_h, km_h
        k.close()
        torch.cuda.empty_cache()
        G_total = WORKLOADS["batched"]["G"]
        r = batched_measure(local, 5, 3, G_total, e2e=False)
        bms = r["total_ms"] / 5
        batched = {"workload": f"{G_total} graphs (n log-uniform 1e3..2e5, avg degree U(4,64), ER or R-MAT)",
                   "graphs_per_s": G_total / (bms / 1e3), "ms_per_batch": bms, "steps": 5, "warmup": 3,
                   "arcs": r["M"], "plain_loop_graphs_per_s": G_total / (r["loop_ms"] / 1e3),
                   "speedup_vs_plain_loop": r["loop_ms"] / bms, "identical_output": r["same"],
                   "autotuned": {key: r["tuning"][key] for key in ("block", "ctas_per_sm", "smem_vertices", "cluster")},
                   "note": "CUDA events around each batched launch; the plain loop is one kcore_decompose per "
                           "graph on the same stream"}
        batched["small_batch"] = small_batch_measure(local)
    served = None
    if args.workload == "rmat24" and ws == 1 and not args.no_served:
        R = WORKLOADS["served"]["requests"]
        runs, serial, _, _ = served_measure(local, R)
        served = {"workload": f"{R} requests, 95% from 256 graphs of the batch distribution, 5% R-MAT scale "
                              "20..24 (edge factor 16), host CSR in and coreness out",
                  "saturation_graphs_per_s": runs[0]["graphs_per_s"],
                  "poisson": [{key: r[key] for key in ("rate", "graphs_per_s", "p50_ms", "p99_ms")} for r in runs[1:]],
                  "serial_plain": {key: serial[key] for key in ("graphs_per_s", "p50_ms", "p99_ms", "rate")},
                  "serial_note": SERIAL_NOTE}
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {
            "workload": workload_name(args.workload, w),
            "n": n, "edges_drawn": E, "undirected_edges": mu, "arcs": m, "kmax": kmax_val,
            "rounds": st["rounds"], "empty_rounds": st["empty_rounds"], "grid": st["grid"],
            "sync_mode": st["sync_mode"], "slice_arcs": st["slice_arcs"], "passes": st["passes"],
            "barriers": st["barriers"], "tail_phases": st["tail_phases"],
            "tail_episodes": st["tail_episodes"],
            **({"sampling": {key: st[key] for key in ("sample_vertices", "sample_recounts", "sample_bag",
                                                       "sample_failed_validations", "sample_heads",
                                                       "sample_reruns")},
                "sample_mu": args.sample_mu, "sample_threshold": args.sample_threshold,
                "sample_check": not args.no_sample_check} if args.sampling else {}),
            **({"warp_combine": True} if args.warp_combine else {}),
            "l2": "inputs larger than L2 and a 258 MB buffer written between timed steps",
            "csr_build_ms": min(csr_ms),
            "csr_build": {"ms": min(csr_ms), "algorithmic_bytes": csr_build_bytes(n, E, m),
                          "achieved_gbs": csr_build_bytes(n, E, m) / (min(csr_ms) / 1e3) / 1e9,
                          "frac": csr_build_bytes(n, E, m) / (min(csr_ms) / 1e3) / 1e9 / peak,
                          "note": "timed apart from the decomposition (a stable LSD radix sort of "
                                  "2E keys, then unique + emit)"},
            "ms_min": min(step_ms), "ms_mean": sum(step_ms) / len(step_ms),
            "parallelism": "replicas" if ws > 1 else "single GPU",
            "wall_s": wall,
        },
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "peak_kind": peak_kind,
                     "algorithmic_bytes": bmin, "kernel": kname},
        "sync_floor_ms": sync_floor["ms"],
        "sync_floor": sync_floor,
        **({"batched": batched} if batched else {}),
        **({"served": served} if served else {}),
        "e2e": e2e,
        # a sampled step is the sampled peel, the two check kernels and the
        # rerun kernel (which returns at once when not needed)
        "gpu_launches": args.steps * (4 if args.sampling and not args.no_sample_check
                                      else 2 if args.sampling else 1),
        "cpu_baseline": cpu,
    }
    clocks = clk.summary()
    if clocks:
        out["clocks"] = clocks
    emit(out)
    if ws > 1:
        dist.barrier()


# ------------------------------------------------------------------ batched
def _batch_inputs(G: int):
    """The batched workload: G graphs, n log-uniform in [1e3, 2e5], average
    degree U(4, 64), ER or R-MAT with probability 1/2 (graph g: seed 5 + g)."""
    import graphgen as gg
    spec = gg.batch_spec(G)
    eoff, s, d = gg.batch_edges(spec)
    gv = np.zeros(G + 1, np.int64)
    np.cumsum(spec[:, 0], out=gv[1:])
    return spec, gv, eoff, s, d


def lpt_partition(weights, parts: int):
    """Greedy longest-processing-time split of independent units over `parts`
    ranks: units by decreasing weight (ties by index), each to the rank with the
    least load so far (ties to the lowest rank). Returns one ascending index
    array per rank; every unit lands in exactly one."""
    import heapq
    w = np.asarray(weights, dtype=np.int64)
    order = sorted(range(len(w)), key=lambda i: (-int(w[i]), i))
    heap = [(0, r) for r in range(parts)]
    out = [[] for _ in range(parts)]
    for i in order:
        load, r = heapq.heappop(heap)
        out[r].append(i)
        heapq.heappush(heap, (load + int(w[i]), r))
    return [np.array(sorted(x), dtype=np.int64) for x in out]


def batch_subset(spec, gv, eoff, s, d, idx):
    """The sub-batch of graphs `idx` (ascending): its spec rows, vertex and edge
    offsets, and edge lists (graph-local ids, so they carry over unchanged)."""
    idx = np.asarray(idx, dtype=np.int64)
    sub = spec[idx]
    gv2 = np.zeros(len(idx) + 1, np.int64)
    np.cumsum(sub[:, 0], out=gv2[1:])
    cnt = eoff[idx + 1] - eoff[idx]
    eoff2 = np.zeros(len(idx) + 1, np.int64)
    np.cumsum(cnt, out=eoff2[1:])
    s2 = np.concatenate([s[eoff[i]:eoff[i + 1]] for i in idx]) if len(idx) else s[:0]
    d2 = np.concatenate([d[eoff[i]:eoff[i + 1]] for i in idx]) if len(idx) else d[:0]
    return sub, gv2, eoff2, s2, d2


def gather_batch_results(core_local, kmax_local, own, gv_global, ws: int, rank: int):
    """Multi-GPU batched run: assembles on rank 0 the coreness of every graph
    of the batch from the ranks' shares. Rank r peeled the graphs own[r]
    (ascending global indices) and holds their coreness concatenated in that
    order (graph-local vertex order) and their k_max. Returns (coreness over
    all vertices of the batch, k_max of every graph) on rank 0, None elsewhere.
    No device collective: host objects are gathered over the process group."""
    import torch.distributed as dist
    parts = [None] * ws if rank == 0 else None
    dist.gather_object((np.asarray(own, np.int64), np.asarray(core_local, np.int32),
                        np.asarray(kmax_local, np.int32)), parts, dst=0)
    if rank != 0:
        return None
    gv = np.asarray(gv_global, np.int64)
    G = len(gv) - 1
    core = np.full(int(gv[-1]), -1, np.int32)
    kmax = np.full(G, -1, np.int32)
    for idx, c, km in parts:
        pos = 0
        for j, g in enumerate(idx):
            n = int(gv[g + 1] - gv[g])
            core[gv[g]:gv[g + 1]] = c[pos:pos + n]
            kmax[g] = km[j]
            pos += n
        if pos != len(c):
            raise ValueError("a rank's coreness does not match its graphs")
    return core, kmax


def small_batch_measure(local: int, G: int = 512, steps: int = 5, warmup: int = 2):
    """The first G graphs of the batched workload, a batch bound by its largest
    graphs: one batched call with the default launch shape (one CTA per graph)
    against the shape the library's autotuner keeps (which may give the largest
    graphs thread-block clusters), both timed with CUDA events, identical
    output checked."""
    import torch

    from paper_2502_08042_gb300 import KCore

    dev = torch.device("cuda", local)
    spec, gv, eoff, s, d = _batch_inputs(G)
    N = int(gv[-1])
    k = KCore(local)
    gvd = torch.from_numpy(gv).to(dev)
    off, adj_buf, m_t = k.build_csr_batched(gvd, torch.from_numpy(eoff).to(dev), torch.from_numpy(s).to(dev),
                                            torch.from_numpy(d).to(dev), int(spec[:, 0].max()), sync=False)
    k.sync()
    M = int(m_t.item())
    adj = adj_buf[:M].clone()
    del adj_buf
    torch.cuda.empty_cache()
    core = torch.empty(N, dtype=torch.int32, device=dev)
    kmax = torch.empty(G, dtype=torch.int32, device=dev)

    def timed():
        for _ in range(warmup):
            k.decompose_batched(gvd, off, adj, core, kmax)
        ts = []
        for _ in range(steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            k.decompose_batched(gvd, off, adj, core, kmax, sync=False)
            e1.record()
            k.sync()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return sum(ts) / len(ts)

    plain_ms = timed()
    ref = core.clone()
    _, _, tuning = k.autotune_batched(gvd, off, adj, core, kmax, repeats=2)
    tuned_ms = timed()
    same = bool(torch.equal(core, ref))
    k.close()
    return {"workload": f"the first {G} graphs of the batched workload", "graphs": G, "arcs": M,
            "ms_one_cta_per_graph": plain_ms, "ms_autotuned": tuned_ms,
            "speedup": plain_ms / tuned_ms, "identical_output": same,
            "autotuned": {key: tuning[key] for key in ("block", "ctas_per_sm", "smem_vertices", "cluster")},
            "note": f"mean of {steps} calls after {warmup} each; one CTA per graph is the default shape"}


def batched_measure(local: int, steps: int, warmup: int, G_total: int, ws: int = 1, rank: int = 0,
                    e2e: bool = True, cluster: int = -1):
    """The batched workload on one GPU: generation, segmented CSR build, the
    library's autotuner (untimed), `steps` timed batched launches after
    `warmup`, then a loop of plain single-graph launches over the same graphs
    (identical output checked) and, with e2e, the end-to-end path from pinned
    host memory. With ws > 1 this rank takes its longest-processing-time share
    of the graphs by arc count. Returns the measurements (times are this
    rank's; the caller reduces over ranks)."""
    import torch

    from paper_2502_08042_gb300 import KCore

    dev = torch.device("cuda", local)
    t0 = time.perf_counter()
    spec, gv, eoff, s, d = _batch_inputs(G_total)
    gv_global, own = gv, None
    if ws > 1:
        # graphs are independent: each rank peels its longest-processing-time
        # share by arc count (strong scaling, no data-path collective)
        own = lpt_partition(eoff[1:] - eoff[:-1], ws)[rank]
        spec, gv, eoff, s, d = batch_subset(spec, gv, eoff, s, d, own)
    G = len(spec)
    gen_s = time.perf_counter() - t0
    N = int(gv[-1])
    k = KCore(local)
    gvd = torch.from_numpy(gv).to(dev)
    eod = torch.from_numpy(eoff).to(dev)
    S = torch.from_numpy(s).to(dev)
    D = torch.from_numpy(d).to(dev)
    del s, d
    # one untimed build first: the handle's first call allocates its workspace
    warm = k.build_csr_batched(gvd, eod, S, D, int(spec[:, 0].max()), sync=False)
    k.sync()
    del warm
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    off, adj_buf, m_t = k.build_csr_batched(gvd, eod, S, D, int(spec[:, 0].max()), sync=False)
    ev1.record()
    k.sync()
    csr_ms = ev0.elapsed_time(ev1)
    M = int(m_t.item())
    adj = adj_buf[:M].clone()
    del adj_buf, S, D, eod
    torch.cuda.empty_cache()
    core = torch.empty(N, dtype=torch.int32, device=dev)
    kmax = torch.empty(G, dtype=torch.int32, device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device=dev)
    if cluster < 0:
        # launch shape picked by the library's autotuner on this batch (untimed)
        t_tune = time.perf_counter()
        _, _, tuning = k.autotune_batched(gvd, off, adj, core, kmax, repeats=2)
        tuning["tune_s"] = time.perf_counter() - t_tune
    else:
        # a fixed shape: the default one, with clusters of `cluster` CTAs for the largest graphs
        k.set_option("batch_cluster", cluster)
        tuning = {"fixed": True, "cluster": cluster}
    for _ in range(warmup):
        k.decompose_batched(gvd, off, adj, core, kmax)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        for i in range(steps):
            flush.zero_()
            evs[i][0].record()
            k.decompose_batched(gvd, off, adj, core, kmax, sync=False)
            evs[i][1].record()
        torch.cuda.synchronize()
    k.sync()
    st = k.stats()
    total_ms = sum(a.elapsed_time(b) for a, b in evs)
    ref = core.clone()
    gathered = None
    if ws > 1:
        # the batch's result assembled on rank 0's host from every rank's share
        res = gather_batch_results(core.cpu().numpy(), kmax.cpu().numpy(), own, gv_global, ws, rank)
        if res is not None:
            gathered = {"vertices": int(len(res[0])), "graphs": int(len(res[1])),
                        "all_assigned": bool((res[1] >= 0).all())}
    # a loop of plain single-graph launches over the same graphs (own handle,
    # workspace sized once for the largest graph)
    offh = off.cpu().numpy()
    kl = KCore(local)
    max_n = int(np.max(np.diff(gv)))
    max_m = int(np.max(offh[gv[1:]] - offh[gv[:-1]]))
    ws_buf = torch.empty(kl.workspace_size(max_n, max_m), dtype=torch.uint8, device=dev)
    kl.set_workspace(ws_buf)
    subs = []
    for g in range(G):
        a, b = int(gv[g]), int(gv[g + 1])
        subs.append((off[a:b + 1] - int(offh[a]), adj[int(offh[a]):int(offh[b])], core[a:b], kmax[g:g + 1]))
    core.fill_(-1)
    for o, a_, c, km in subs[:64]:
        kl.decompose(o.contiguous(), a_, c, km, sync=False)
    kl.sync()
    torch.cuda.synchronize()
    core.fill_(-1)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    subs = [(o.contiguous(), a_, c, km) for o, a_, c, km in subs]
    torch.cuda.synchronize()
    e0.record()
    for o, a_, c, km in subs:
        kl.decompose(o, a_, c, km, sync=False)
    e1.record()
    kl.sync()
    loop_ms = e0.elapsed_time(e1)
    same = bool(torch.equal(core, ref))
    del subs, ws_buf
    kl.close()
    e2e_ms = []
    if e2e:
        # end to end: segmented CSR from pinned host memory, coreness back
        gv_h = torch.from_numpy(gv).pin_memory()
        off_h = off.cpu().pin_memory()
        adj_h = adj.cpu().pin_memory()
        core_h = torch.empty(N, dtype=torch.int32, pin_memory=True)
        km_h = torch.empty(G, dtype=torch.int32, pin_memory=True)
        for it in range(3):
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            gvd2 = gv_h.to(dev, non_blocking=True)
            off2 = off_h.to(dev, non_blocking=True)
            adj2 = adj_h.to(dev, non_blocking=True)
            c2, k2 = k.decompose_batched(gvd2, off2, adj2, sync=False)
            core_h.copy_(c2, non_blocking=True)
            km_h.copy_(k2, non_blocking=True)
            k.sync()
            torch.cuda.synchronize()
            e2e_ms.append((time.perf_counter() - t1) * 1e3)
            del gvd2, off2, adj2, c2, k2
    k.close()
    del off, adj, core, kmax, flush, gvd
    torch.cuda.empty_cache()
    return dict(spec=spec, gv=gv, G=G, N=N, M=M, gen_s=gen_s, csr_ms=csr_ms, tuning=tuning, grid=st["grid"],
                total_ms=total_ms, loop_ms=loop_ms, same=same, e2e_ms=e2e_ms, clocks=clk.summary(),
                gathered=gathered)


def run_batched(args):
    import torch
    import torch.distributed as dist

    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    G_total = args.graphs or WORKLOADS["batched"]["G"]
    r = batched_measure(local, args.steps, args.warmup, G_total, ws, rank, cluster=args.batch_cluster)
    ms = max_over_ranks(r["total_ms"], ws, dev) / args.steps
    e2e_best = max_over_ranks(min(r["e2e_ms"][1:]), ws, dev)
    if rank != 0:
        if ws > 1:
            dist.barrier()
        return
    G, N, M = r["G"], r["N"], r["M"]
    peak, peak_kind = load_peaks()
    bmin = 8 * (N + G) + 4 * M + 12 * N
    achieved = bmin / (ms / 1e3) / 1e9
    cpu = None if args.no_cpu_baseline else cpu_batch_baseline(r["spec"], r["gv"], G)
    out = {
        "metric": METRIC, "value": G_total / (ms / 1e3), "unit": "graphs/s", "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "strong" if ws > 1 else "weak", "vs_baseline": None, "dtype": "int32",
        "data": "synthetic",
        "config": {"workload": f"batched: {G_total} graphs (n log-uniform 1e3..2e5, avg degree U(4,64), "
                               "ER or R-MAT)", "graphs": G_total, "graphs_rank0": G, "vertices_rank0": N,
                   "arcs_rank0": M,
                   "parallelism": (f"graphs split over {ws} GPUs by arc count (longest processing "
                                   "time first); the job's time is the slowest rank's") if ws > 1
                   else "single GPU",
                   "undirected_edges_per_s_rank0": M / 2 / (ms / 1e3), "csr_build_ms": r["csr_ms"],
                   "generation_s": r["gen_s"], "grid": r["grid"], "autotuned": r["tuning"],
                   "l2": "inputs larger than L2 and a 258 MB buffer written between timed steps"},
        "plain_loop": {"graphs_per_s": G / (r["loop_ms"] / 1e3), "ms": r["loop_ms"],
                       "identical_output": r["same"], "speedup": r["loop_ms"] / ms},
        **({"gathered_on_host": r["gathered"]} if r["gathered"] else {}),
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None, "peak_kind": peak_kind,
                     "algorithmic_bytes": bmin, "kernel": "batch_peel"},
        "e2e": {"value": G_total / (e2e_best / 1e3), "unit": "graphs/s",
                "h2d_bytes_per_step": 8 * (G + 1) + 8 * (N + 1) + 4 * M,
                "d2h_bytes_per_step": 4 * N + 4 * G, "ms_per_step": e2e_best},
        "gpu_launches": 2 * args.steps,
        "cpu_baseline": cpu,
    }
    if r["clocks"]:
        out["clocks"] = r["clocks"]
    emit(out)
    if ws > 1:
        dist.barrier()


def cpu_batch_baseline(spec, gv, G, sample: int = 256):
    """The oracle (per-graph Batagelj-Zaversnik) on a sample of the batch,
    graphs spread over all host cores."""
    import graphgen as gg
    import oracle
    idx = np.linspace(0, G - 1, min(sample, G)).astype(int)
    sub = spec[idx]
    eoff, s, d = gg.batch_edges(sub)
    ns = sub[:, 0]
    gvs = np.zeros(len(idx) + 1, np.int64)
    np.cumsum(ns, out=gvs[1:])
    offs, adjs, base = [], [], 0
    for g in range(len(idx)):
        o, a = oracle.build_csr(int(ns[g]), s[eoff[g]:eoff[g + 1]], d[eoff[g]:eoff[g + 1]])
        offs.append(o[:-1] + base)
        adjs.append(a)
        base += len(a)
    off = np.concatenate(offs + [np.array([base], np.int64)])
    adj = np.concatenate(adjs)
    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    oracle.bz_batch(gvs, off, adj, threads=threads)
    t = time.perf_counter() - t0
    return {"value": len(idx) / t, "unit": "graphs/s", "cores": threads, "kind": "oracle",
            "sample": f"{len(idx)} graphs of the batch (every {G // len(idx)}th), per-graph "
                      f"Batagelj-Zaversnik on {threads} host threads, {t:.2f} s"}


# ------------------------------------------------------------------ served
SERIAL_NOTE = ("serial plain launches (kcore_decompose_host per request): each service time measured back to "
               "back, then placed on the same arrival timeline (a request starts at its arrival or when the "
               "previous one finishes); arrivals are not replayed")


def served_measure(local: int, R: int, batch_cluster: int = 0):
    """The served workload on one GPU: R requests (95% drawn from 256 graphs of
    the batch distribution, 5% from one R-MAT graph per scale 20..24) through a
    KCoreServer, all at once (saturation) and as Poisson arrivals at 0.5x and
    0.8x the saturation rate; then serial plain launches over the same
    requests. batch_cluster: the server's clusters for the largest graphs of a
    batched launch (0: its default; 1: one CTA per graph). Returns (runs,
    serial, h2d bytes, d2h bytes)."""
    import torch

    import graphgen as gg
    from paper_2502_08042_gb300 import KCore, KCoreServer

    dev = torch.device("cuda", local)
    rng = np.random.default_rng(11)
    k = KCore(local)
    # distinct graphs: 256 from the batch distribution, one R-MAT per scale 20..24
    spec, gv, eoff, s, d = _batch_inputs(256)
    offd, adjd = k.build_csr_batched(torch.from_numpy(gv).to(dev), torch.from_numpy(eoff).to(dev),
                                     torch.from_numpy(s).to(dev), torch.from_numpy(d).to(dev),
                                     int(spec[:, 0].max()))
    offh = offd.cpu().numpy()
    adjh = adjd.cpu().numpy()
    graphs = []
    for g in range(256):
        a, b = int(gv[g]), int(gv[g + 1])
        o = offh[a:b + 1] - offh[a]
        graphs.append((torch.from_numpy(o.copy()).pin_memory().numpy(),
                       torch.from_numpy(adjh[offh[a]:offh[b]].copy()).pin_memory().numpy()))
    large = []
    for sc in range(20, 25):
        rs, rd = gg.rmat(sc, 16, seed=100 + sc, perm_seed=200 + sc)
        o, a = k.build_csr(1 << sc, torch.from_numpy(rs).to(dev), torch.from_numpy(rd).to(dev))
        large.append((o.cpu().pin_memory().numpy(), a.cpu().pin_memory().numpy()))
        del rs, rd, o, a
    torch.cuda.empty_cache()
    kinds = rng.random(R) < 0.05
    which = np.where(kinds, rng.integers(0, 5, R), rng.integers(0, 256, R))
    reqs = [large[w] if kd else graphs[w] for kd, w in zip(kinds, which)]
    outs = [torch.empty(max(len(o) - 1, 1), dtype=torch.int32, pin_memory=True).numpy() for o, _ in reqs]

    def serve(rate):
        """Poisson arrivals at `rate` requests/s (inf: all at once)."""
        gaps = rng.exponential(1.0 / rate, R) if np.isfinite(rate) else np.zeros(R)
        arrive = np.cumsum(gaps)
        done_t = np.zeros(R)
        with KCoreServer(local, pool_bytes=48 << 30, batch_cluster=batch_cluster) as srv:
            tick = {}
            nxt = 0
            t0 = time.perf_counter()
            while len(tick) or nxt < R:
                now = time.perf_counter() - t0
                while nxt < R and arrive[nxt] <= now:
                    o, a = reqs[nxt]
                    t = srv.submit(o, a, outs[nxt])
                    if t is None:
                        break
                    tick[t] = nxt
                    nxt += 1
                for t, km, stt in srv.poll():
                    i = tick.pop(t)
                    done_t[i] = time.perf_counter() - t0
                    if stt != 0:
                        raise RuntimeError(f"request {i} failed with status {stt}")
            total = time.perf_counter() - t0
        lat = (done_t - arrive) * 1e3
        return {"rate": rate if np.isfinite(rate) else "all at t=0", "graphs_per_s": R / total,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "wall_s": total}

    serve(float("inf"))  # warm-up
    sat = serve(float("inf"))
    runs = [sat]
    for frac in (0.5, 0.8):
        runs.append(serve(frac * sat["graphs_per_s"]))
    # serial plain launches: one request at a time, host arrays in and out
    rate = runs[-1]["rate"]
    gaps = rng.exponential(1.0 / rate, R)
    arrive = np.cumsum(gaps)
    biggest = max(range(R), key=lambda i: len(reqs[i][1]))
    o0, a0 = reqs[biggest]
    k.decompose_host_into(o0, a0, outs[biggest], np.zeros(1, np.int32))
    start = np.zeros(R)
    fin = np.zeros(R)
    busy = 0.0
    km = np.zeros(1, np.int32)
    t0 = time.perf_counter()
    for i in range(R):
        o, a = reqs[i]
        t1 = time.perf_counter()
        k.decompose_host_into(o, a, outs[i], km)
        dt = time.perf_counter() - t1
        start[i] = max(arrive[i], fin[i - 1] if i else 0.0)
        fin[i] = start[i] + dt
        busy += dt
    lat = (fin - arrive) * 1e3
    serial = {"graphs_per_s": R / busy, "p50_ms": float(np.percentile(lat, 50)),
              "p99_ms": float(np.percentile(lat, 99)), "rate": rate, "note": SERIAL_NOTE}
    h2d = int(sum(8 * len(o) + 4 * len(a) for o, a in reqs))
    d2h = int(sum(4 * (len(o) - 1) + 4 for o, _ in reqs))
    k.close()
    del graphs, large, reqs, outs
    torch.cuda.empty_cache()
    return runs, serial, h2d, d2h


def run_served(args):
    import torch

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    R = WORKLOADS["served"]["requests"]
    # --batch-cluster: 0 = one CTA per graph (the server's 1), C = clusters of C, unset = the server's default
    cluster = 0 if args.batch_cluster < 0 else (1 if args.batch_cluster == 0 else args.batch_cluster)
    runs, serial, h2d, d2h = served_measure(local, R, cluster)
    sat = runs[0]
    out = {
        "metric": METRIC, "value": sat["graphs_per_s"], "unit": "graphs/s", "n_gpus": 1,
        "steps": 1, "warmup": 1, "ms_per_step": sat["wall_s"] * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": {"workload": f"served: {R} requests, 95% from the batch distribution (256 distinct "
                               "graphs), 5% R-MAT scale 20..24; Poisson arrivals",
                   "requests": R},
        "served": runs, "serial_plain": serial,
        "e2e": {"value": sat["graphs_per_s"], "unit": "graphs/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": None,
    }
    emit(out)


# single-graph schedule (stats "sync_mode") -> (kernel name, its source file)
PEEL_KERNELS = {1: ("peel_persistent", "peel.cu"), 2: ("peel_bsp", "peel_bsp.cu"), 3: ("peel_bsp", "peel_bsp.cu")}


def kernel_revision(src: str = "peel_bsp.cu") -> str:
    """Hash of a peel kernel source and the header of its shared layout and
    defaults, to tie recorded ncu traffic to them."""
    import hashlib
    h = hashlib.sha1()
    for name in (src, "kcore_peel.h"):
        with open(os.path.join(ROOT, "paper_2502_08042_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:12]


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--workload", default="rmat24", choices=sorted(WORKLOADS))
    ap.add_argument("--sampling", action="store_true",
                    help="single-graph workloads: the sampled peel of Algorithms 4-5 (mode 2)")
    ap.add_argument("--sample-mu", type=int, default=0, help="heads per sampling period (0 = auto)")
    ap.add_argument("--sample-threshold", type=int, default=-1, help="sampling degree threshold (-1 = auto)")
    ap.add_argument("--no-sample-check", action="store_true", help="skip the final check of a sampled run")
    ap.add_argument("--warp-combine", action="store_true",
                    help="single-graph workloads: warp-aggregated decrements (mode 2)")
    ap.add_argument("--sync-mode", type=int, default=0, choices=[0, 1, 2, 3],
                    help="single-graph schedule (0: the library's default)")
    ap.add_argument("--batch-cluster", type=int, default=-1, choices=[-1, 0, 2, 4, 8],
                    help="batched workload: skip the autotuner and run the default shape with clusters of "
                         "this many CTAs for the largest graphs (0: one CTA per graph); served workload: the "
                         "server's clusters for its batched launches (0: one CTA per graph)")
    ap.add_argument("--graphs", type=int, default=0,
                    help="batched workload: first G graphs of the distribution (default 4096; "
                         "smaller batches are for profiling)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true",
                    help="default workload: skip the batched sub-record measured after the main line")
    ap.add_argument("--no-served", action="store_true",
                    help="default workload: skip the served sub-record measured after the main line")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "kquery":
        run_kquery(args)
    elif args.workload == "served":
        run_served(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
