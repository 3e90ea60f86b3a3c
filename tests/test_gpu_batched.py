"""Parity of the batched peel and the batched CSR build (through the C ABI)
with the CPU oracle: bit-exact coreness and k_max per graph, under every launch
shape (shared-memory or global induced degrees, block sizes), with empty and
isolated-only graphs in the batch."""
import numpy as np
import pytest

import graphgen as gg
import oracle
from tests.batch_util import oracle_segmented, spec_batch

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2502_08042_gb300 import KCore  # noqa: E402


def _t(x, dtype):
    return torch.from_numpy(np.ascontiguousarray(x, dtype)).cuda()


def run_batched(k, gv, off, adj):
    core, km = k.decompose_batched(_t(gv, np.int64), _t(off, np.int64), _t(adj, np.int32))
    return core.cpu().numpy(), km.cpu().numpy()


def check_batch(k, gv, off, adj):
    want_core, want_km = oracle.bz_batch(gv, off, adj)
    core, km = run_batched(k, gv, off, adj)
    np.testing.assert_array_equal(core, want_core)
    np.testing.assert_array_equal(km, want_km)


@pytest.fixture(scope="module")
def small_batch():
    spec, eoff, s, d, ns, lists = spec_batch(48, nmin=50, nmax=6000, seed=21)
    return oracle_segmented(ns, lists)


@pytest.mark.parametrize("opts", [
    dict(), dict(batch_smem_vertices=0), dict(batch_smem_vertices=500), dict(batch_block=256),
    dict(batch_block=1024), dict(batch_block=1024, batch_ctas_per_sm=1),
    dict(batch_block=256, batch_ctas_per_sm=8, batch_smem_vertices=2000),
])
def test_batched_launch_shapes(small_batch, opts):
    gv, off, adj = small_batch
    with KCore(0, **opts) as k:
        check_batch(k, gv, off, adj)


def test_batched_with_empty_and_isolated_graphs():
    parts = [gg.complete(30), (0, np.zeros(0, np.int32), np.zeros(0, np.int32)), gg.path(1000),
             (17, np.zeros(0, np.int32), np.zeros(0, np.int32)), gg.staircase(90), gg.star(3000),
             (0, np.zeros(0, np.int32), np.zeros(0, np.int32)), gg.grid2d(40, 40)]
    ns = [p[0] for p in parts]
    gv, off, adj = oracle_segmented(ns, [(p[1], p[2]) for p in parts])
    with KCore(0) as k:
        check_batch(k, gv, off, adj)
        core, km = run_batched(k, gv, off, adj)
        assert km[1] == 0 and km[3] == 0 and km[6] == 0


def test_batched_matches_single_graph_calls():
    spec, eoff, s, d, ns, lists = spec_batch(12, nmin=2000, nmax=60000, seed=33)
    gv, off, adj = oracle_segmented(ns, lists)
    with KCore(0) as k:
        core, km = run_batched(k, gv, off, adj)
        for g in range(len(ns)):
            a, b = gv[g], gv[g + 1]
            o = off[a:b + 1] - off[a]
            ad = adj[off[a]:off[b]]
            c1, k1 = k.decompose(_t(o, np.int64), _t(ad, np.int32))
            np.testing.assert_array_equal(core[a:b], c1.cpu().numpy())
            assert km[g] == int(k1.item())


def test_batched_workload_sample():
    """A sample of the batched workload at full per-graph sizes (n up to 2e5)."""
    spec, eoff, s, d, ns, lists = spec_batch(64, seed=5)
    gv, off, adj = oracle_segmented(ns, lists)
    with KCore(0) as k:
        check_batch(k, gv, off, adj)


@pytest.mark.parametrize("seed", [5, 77])
def test_batched_csr_build_matches_oracle(seed):
    spec, eoff, s, d, ns, lists = spec_batch(40, nmin=100, nmax=30000, seed=seed)
    # add duplicates, reversed pairs and self-loops to every graph
    lists2, eo = [], [0]
    for (ss, dd), n in zip(lists, ns):
        rng = np.random.default_rng(int(n))
        extra = rng.integers(0, n, (n // 3 + 1, 2)).astype(np.int32)
        ss2 = np.concatenate([ss, dd[: len(dd) // 4], extra[:, 0], extra[:5, 0]])
        dd2 = np.concatenate([dd, ss[: len(ss) // 4], extra[:, 1], extra[:5, 0]])
        lists2.append((ss2, dd2))
        eo.append(eo[-1] + len(ss2))
    gv, off, adj = oracle_segmented(ns, lists2)
    S = np.concatenate([x[0] for x in lists2])
    D = np.concatenate([x[1] for x in lists2])
    with KCore(0) as k:
        o2, a2 = k.build_csr_batched(_t(gv, np.int64), _t(np.array(eo), np.int64), _t(S, np.int32),
                                     _t(D, np.int32), max(ns))
        np.testing.assert_array_equal(o2.cpu().numpy(), off)
        np.testing.assert_array_equal(a2.cpu().numpy(), adj)
        check_batch(k, gv, off, adj)


def test_batched_csr_rejects_foreign_ids():
    from paper_2502_08042_gb300 import KCoreError
    gv = _t(np.array([0, 3, 5]), np.int64)
    eo = _t(np.array([0, 1, 2]), np.int64)
    S = _t(np.array([0, 0]), np.int32)
    D = _t(np.array([1, 4]), np.int32)  # 4 is outside the second graph (2 vertices)
    with KCore(0) as k:
        with pytest.raises(KCoreError) as e:
            k.build_csr_batched(gv, eo, S, D, 3)
        assert e.value.code == "INVALID"


def test_batched_regression_frontier_visibility():
    """64 copies of one R-MAT graph of the batched workload (n = 6937, with
    isolated vertices) whose frontier selection almost fills a scan tile:
    every copy must come out exactly as the oracle, on repeated runs."""
    spec = gg.batch_spec(4096)
    n, m, kind, sd = [int(x) for x in spec[640]]
    s, d = gg.rmat_n(n, m, seed=sd)
    off, adj = oracle.build_csr(n, s, d)
    want = oracle.bz(n, off, adj)
    copies = 64
    gv = np.arange(copies + 1, dtype=np.int64) * n
    offs = np.concatenate([off[:-1] + i * len(adj) for i in range(copies)] +
                          [np.array([copies * len(adj)], np.int64)])
    adjs = np.tile(adj, copies)
    with KCore(0) as k:
        for _ in range(3):
            core, km = run_batched(k, gv, offs, adjs)
            np.testing.assert_array_equal(core.reshape(copies, n), np.broadcast_to(want, (copies, n)))
            assert (km == want.max()).all()


@pytest.mark.slow
def test_batched_full_workload_matches_oracle():
    """All 4,096 graphs of the batched workload (5.3 G arcs): the batched CSR
    build and the batched peel against the oracle, graph by graph."""
    import os
    from concurrent.futures import ThreadPoolExecutor
    G = 4096
    spec = gg.batch_spec(G)
    eoff, s, d = gg.batch_edges(spec)
    gv = np.zeros(G + 1, np.int64)
    np.cumsum(spec[:, 0], out=gv[1:])
    want = [None] * G

    def one(g):
        o, a = oracle.build_csr(int(spec[g, 0]), s[eoff[g]:eoff[g + 1]], d[eoff[g]:eoff[g + 1]])
        want[g] = oracle.bz(len(o) - 1, o, a)

    with ThreadPoolExecutor(os.cpu_count()) as ex:
        list(ex.map(one, range(G)))
    with KCore(0) as k:
        gvd = _t(gv, np.int64)
        off, adj = k.build_csr_batched(gvd, _t(eoff, np.int64), _t(s, np.int32), _t(d, np.int32),
                                       int(spec[:, 0].max()))
        core, km = k.decompose_batched(gvd, off, adj)
        core = core.cpu().numpy()
        km = km.cpu().numpy()
    bad = [g for g in range(G) if not np.array_equal(core[gv[g]:gv[g + 1]], want[g])]
    assert bad == []
    assert all(km[g] == want[g].max() for g in range(G))


def test_autotune_picks_a_shape_and_stays_exact(small_batch):
    """The autotuner times the launch shapes on the batch, keeps the fastest
    in the handle's options, and every result along the way stays exact."""
    gv, off, adj = small_batch
    want_core, want_km = oracle.bz_batch(gv, off, adj)
    with KCore(0) as k:
        core, km, t = k.autotune_batched(_t(gv, np.int64), _t(off, np.int64), _t(adj, np.int32), repeats=1)
        np.testing.assert_array_equal(core.cpu().numpy(), want_core)
        np.testing.assert_array_equal(km.cpu().numpy(), want_km)
        assert t["block"] in (256, 512, 1024) and t["candidates"] >= 2 and t["ms"] > 0
        assert k.get_option("batch_block") == t["block"]
        assert k.get_option("batch_ctas_per_sm") == t["ctas_per_sm"]
        assert k.stats()["batch_block"] == t["block"]
        check_batch(k, gv, off, adj)  # later calls run the tuned shape


def _relabel(ns, lists, seed):
    """Each graph with its vertex ids permuted: the same sizes, another CSR."""
    rng = np.random.default_rng(seed)
    out = []
    for n, (s, d) in zip(ns, lists):
        p = rng.permutation(n).astype(np.int32)
        out.append((p[s], p[d]))
    return out


def test_batched_call_captured_in_cuda_graph():
    """A batched call captured in a CUDA graph replays exactly, also after the
    input buffers were refilled with other graphs of the same sizes."""
    spec, eoff, s, d, ns, lists = spec_batch(32, nmin=50, nmax=4000, seed=33)
    gv, off, adj = oracle_segmented(ns, lists)
    gv2, off2, adj2 = oracle_segmented(ns, _relabel(ns, lists, 9))
    assert len(adj2) == len(adj) and (gv2 == gv).all()
    want1, km1 = oracle.bz_batch(gv, off, adj)
    want2, km2 = oracle.bz_batch(gv2, off2, adj2)
    with KCore(0) as k:
        dgv, doff, dadj = _t(gv, np.int64), _t(off, np.int64), _t(adj, np.int32)
        core = torch.empty(int(gv[-1]), dtype=torch.int32, device="cuda:0")
        km = torch.empty(len(ns), dtype=torch.int32, device="cuda:0")
        k.decompose_batched(dgv, doff, dadj, core, km)  # sizes the workspace outside the capture
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            k.decompose_batched(dgv, doff, dadj, core, km, sync=False)
        for o, a, want, wkm in [(off, adj, want1, km1), (off2, adj2, want2, km2)]:
            doff.copy_(_t(o, np.int64))
            dadj.copy_(_t(a, np.int32))
            core.fill_(-7)
            km.fill_(-7)
            graph.replay()
            torch.cuda.synchronize()
            k.sync()
            np.testing.assert_array_equal(core.cpu().numpy(), want)
            np.testing.assert_array_equal(km.cpu().numpy(), wkm)
