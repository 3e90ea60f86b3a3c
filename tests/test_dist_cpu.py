"""The multi-process path of bench.py on the CPU: two gloo ranks (replicas,
weak scaling) agree on the slowest rank's time and on the job's throughput;
the batched workload splits its graphs over ranks by arc count."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        w, r, loc = bench.dist_env()
        my_ms = 10.0 + 5.0 * rank  # rank 1 is slower
        mx = bench.max_over_ranks(my_ms, w)
        value = bench.job_throughput(1e9, w, mx)
        out.put((r, w, loc, mx, value))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, ws, port, out)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, *_ in res] == [0, 1]
    for r, w, loc, mx, value in res:
        assert w == 2 and loc == r
        assert mx == 15.0                    # the slowest rank's time, on every rank
        assert value == pytest.approx(2 * 1e9 / 0.015)  # two replicas in that time


def test_single_process_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert bench.job_throughput(3e9, 1, 1000.0) == pytest.approx(3e9)


def _shard_rank(rank, ws, port, G, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        spec, gv, eoff, s, d = bench._batch_inputs(G)
        own = bench.lpt_partition(eoff[1:] - eoff[:-1], ws)[rank]
        sub, gv2, eoff2, s2, d2 = bench.batch_subset(spec, gv, eoff, s, d, own)
        # each rank peels its share; the job's time is the slowest rank's
        load = int(eoff2[-1])
        mx = bench.max_over_ranks(float(load), ws)
        out.put((rank, own.tolist(), load, mx))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_batched_graphs_split_over_two_gloo_ranks():
    """The batched workload over two ranks: every graph lands on exactly one
    rank, the split is balanced by arc count, and both ranks agree on the
    slowest share (no data-path collective: only the timing reduction)."""
    ws, port, G = 2, _free_port(), 24
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_shard_rank, args=(r, ws, port, G, out)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=300) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    owned = sorted(g for _, own, _, _ in res for g in own)
    assert owned == list(range(G))
    loads = [load for _, _, load, _ in res]
    assert all(mx == max(loads) for *_, mx in res)
    sys.path.insert(0, ROOT)
    import bench
    spec, gv, eoff, s, d = bench._batch_inputs(G)
    w = eoff[1:] - eoff[:-1]
    assert max(loads) - min(loads) <= int(w.max())  # LPT: within one unit of balance


def test_lpt_partition_and_subset():
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    w = np.array([5, 9, 1, 7, 7, 3, 0, 2], dtype=np.int64)
    parts = bench.lpt_partition(w, 3)
    assert sorted(np.concatenate(parts).tolist()) == list(range(len(w)))
    assert all((np.diff(p) > 0).all() for p in parts)
    loads = sorted(int(w[p].sum()) for p in parts)
    assert loads == [11, 11, 12]  # 9+2+0 | 7+3+1 | 7+5 by longest processing time first
    assert [len(p) for p in bench.lpt_partition(w, 1)] == [len(w)]
    spec, gv, eoff, s, d = bench._batch_inputs(6)
    idx = np.array([1, 4, 5])
    sub, gv2, eoff2, s2, d2 = bench.batch_subset(spec, gv, eoff, s, d, idx)
    assert (sub == spec[idx]).all()
    assert (np.diff(gv2) == np.diff(gv)[idx]).all()
    for j, g in enumerate(idx):
        np.testing.assert_array_equal(s2[eoff2[j]:eoff2[j + 1]], s[eoff[g]:eoff[g + 1]])
        np.testing.assert_array_equal(d2[eoff2[j]:eoff2[j + 1]], d[eoff[g]:eoff[g + 1]])


def _gather_rank(rank, ws, port, G, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(ws), RANK=str(rank),
                      LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    import oracle
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        spec, gv, eoff, s, d = bench._batch_inputs(G)
        own = bench.lpt_partition(eoff[1:] - eoff[:-1], ws)[rank]
        sub, gv2, eoff2, s2, d2 = bench.batch_subset(spec, gv, eoff, s, d, own)
        # this rank's share peeled by the oracle, graph by graph
        cores, kms = [], []
        for j in range(len(own)):
            n = int(gv2[j + 1] - gv2[j])
            off, adj = oracle.build_csr(n, s2[eoff2[j]:eoff2[j + 1]], d2[eoff2[j]:eoff2[j + 1]])
            c = oracle.bz(n, off, adj)
            cores.append(c)
            kms.append(int(c.max()) if n else 0)
        core = np.concatenate(cores) if cores else np.zeros(0, np.int32)
        res = bench.gather_batch_results(core, np.array(kms, np.int32), own, gv, ws, rank)
        out.put((rank, None if res is None else (res[0].tolist(), res[1].tolist())))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_batched_results_gathered_on_rank_0():
    """Two gloo ranks each peel their longest-processing-time share of a batch;
    rank 0 assembles the coreness of every graph in the batch's own vertex
    order, equal to peeling the whole batch in one process."""
    ws, port, G = 2, _free_port(), 10
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    procs = [ctx.Process(target=_gather_rank, args=(r, ws, port, G, out)) for r in range(ws)]
    for p in procs:
        p.start()
    res = dict(out.get(timeout=300) for _ in range(ws))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[1] is None and res[0] is not None
    sys.path.insert(0, ROOT)
    import numpy as np
    import bench
    import oracle
    spec, gv, eoff, s, d = bench._batch_inputs(G)
    want, want_km = [], []
    for g in range(G):
        n = int(gv[g + 1] - gv[g])
        off, adj = oracle.build_csr(n, s[eoff[g]:eoff[g + 1]], d[eoff[g]:eoff[g + 1]])
        c = oracle.bz(n, off, adj)
        want.append(c)
        want_km.append(int(c.max()) if n else 0)
    core, km = res[0]
    np.testing.assert_array_equal(np.array(core, np.int32), np.concatenate(want))
    assert km == want_km
