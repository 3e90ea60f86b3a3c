"""The clustered form of the batched peel (KCORE_OPT_BATCH_CLUSTER): graphs
with at least KCORE_OPT_BATCH_BIG_ARCS arcs are peeled by a thread-block
cluster of 2, 4 or 8 CTAs, the others by one CTA each. Coreness and k_max must
equal the oracle's bit for bit under every cluster and block size, with the
threshold forcing nearly every graph onto clusters and with the default
threshold, on batches mixing a few large graphs with many small, empty and
edgeless ones; a malformed graph must be reported without upsetting the rest."""
import numpy as np
import pytest

import graphgen as gg
import oracle
from tests.batch_util import oracle_segmented, spec_batch

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2502_08042_gb300 import KCore, KCoreError  # noqa: E402


def _t(x, dtype):
    return torch.from_numpy(np.ascontiguousarray(x, dtype)).cuda()


def _run(k, gv, off, adj):
    core, km = k.decompose_batched(_t(gv, np.int64), _t(off, np.int64), _t(adj, np.int32))
    return core.cpu().numpy(), km.cpu().numpy()


@pytest.fixture(scope="module")
def mixed_batch():
    """Three large graphs (an R-MAT graph of 2^15 vertices, a star of 40,000
    leaves, a staircase under a clique of 300) among 40 graphs of the batched
    workload's distribution, a 3D grid, an empty and an edgeless graph."""
    _, _, _, _, ns, lists = spec_batch(40, nmin=50, nmax=5000, seed=31)
    s, d = gg.rmat(15, 16, seed=9, perm_seed=10)
    big = [(1 << 15, s, d), gg.star(40000), gg.staircase(300), gg.grid3d(12, 12, 12)]
    empty = [(0, np.zeros(0, np.int32), np.zeros(0, np.int32)), (500, np.zeros(0, np.int32), np.zeros(0, np.int32))]
    parts = [(n, (a, b)) for n, a, b in big + empty] + list(zip(ns, lists))
    order = np.random.default_rng(3).permutation(len(parts))
    parts = [parts[i] for i in order]
    gv, off, adj = oracle_segmented([p[0] for p in parts], [p[1] for p in parts])
    want_core, want_km = oracle.bz_batch(gv, off, adj)
    return gv, off, adj, want_core, want_km


@pytest.mark.parametrize("block", [512, 1024])
@pytest.mark.parametrize("cluster", [2, 4, 8])
@pytest.mark.parametrize("big_arcs", [1, 0])
def test_clustered_matches_oracle(mixed_batch, block, cluster, big_arcs):
    gv, off, adj, want_core, want_km = mixed_batch
    with KCore(0, batch_block=block, batch_cluster=cluster, batch_big_arcs=big_arcs) as k:
        for _ in range(2):
            core, km = _run(k, gv, off, adj)
            np.testing.assert_array_equal(core, want_core)
            np.testing.assert_array_equal(km, want_km)
        assert k.stats()["batch_cluster"] == cluster


def test_clustered_regression_frontier_visibility():
    """64 copies of one graph of the batched workload, every copy on a cluster
    of 8 CTAs: frontiers and active lists written by one CTA and read by the
    others after the cluster barrier, on repeated runs."""
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
    with KCore(0, batch_cluster=8, batch_big_arcs=1) as k:
        for _ in range(3):
            core, km = _run(k, gv, offs, adjs)
            np.testing.assert_array_equal(core.reshape(copies, n), np.broadcast_to(want, (copies, n)))
            assert (km == want.max()).all()


def test_clustered_reports_a_malformed_graph():
    """A large graph whose offsets run backwards is reported (NOT_SIMPLE,
    k_max -1) by the cluster peeling it; the handle then peels a sound batch."""
    parts = [gg.complete(200), gg.path(3000), gg.star(5000)]
    gv, off, adj = oracle_segmented([p[0] for p in parts], [(p[1], p[2]) for p in parts])
    bad = off.copy()
    bad[gv[0] + 10] = bad[gv[0] + 11] + 5  # vertex 10 of the clique: offsets decrease
    with KCore(0, batch_cluster=4, batch_big_arcs=1) as k:
        with pytest.raises(KCoreError) as e:
            _run(k, gv, bad, adj)
        assert e.value.code == "NOT_SIMPLE"
        want_core, want_km = oracle.bz_batch(gv, off, adj)
        core, km = _run(k, gv, off, adj)
        np.testing.assert_array_equal(core, want_core)
        np.testing.assert_array_equal(km, want_km)


def test_cluster_options_are_checked():
    with KCore(0) as k:
        for bad in (1, 3, 16, -1):
            with pytest.raises(KCoreError):
                k.set_option("batch_cluster", bad)
        with pytest.raises(KCoreError):
            k.set_option("batch_big_arcs", -5)
        k.set_option("batch_cluster", 4)
        k.set_option("batch_block", 256)
        parts = [gg.complete(20), gg.path(50)]
        gv, off, adj = oracle_segmented([p[0] for p in parts], [(p[1], p[2]) for p in parts])
        with pytest.raises(KCoreError) as e:
            _run(k, gv, off, adj)
        assert e.value.code == "INVALID"


def test_autotuner_times_the_clustered_form_and_stays_exact(mixed_batch):
    """The batched autotuner's candidates include the clustered form; whatever
    it keeps, the result stays exact and the handle's options hold its choice."""
    gv, off, adj, want_core, want_km = mixed_batch
    with KCore(0) as k:
        core, km, t = k.autotune_batched(_t(gv, np.int64), _t(off, np.int64), _t(adj, np.int32), repeats=1)
        np.testing.assert_array_equal(core.cpu().numpy(), want_core)
        np.testing.assert_array_equal(km.cpu().numpy(), want_km)
        assert t["candidates"] >= 14
        assert t["cluster"] in (0, 2, 4, 8)
        assert k.get_option("batch_cluster") == t["cluster"]
        assert k.get_option("batch_big_arcs") == 0
        core, km = _run(k, gv, off, adj)
        np.testing.assert_array_equal(core, want_core)
