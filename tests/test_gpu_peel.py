"""Parity of the GPU peel (through the C ABI) with the CPU oracle: bit-exact
coreness on closed forms, hand-derived fixtures, random graphs over many seeds,
the ER n=10,000 workload, adversarial shapes and every tuning mode, in all
schedules (1: asynchronous, 2: bulk-synchronous with grid barriers, 3: the
offline peel of Algorithm 2 on the same kernel)."""
import numpy as np
import pytest

import graphgen as gg
import oracle
from tests import golden_io

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2502_08042_gb300 import KCore, KCoreError  # noqa: E402
from tests.gpu_util import assert_parity, gpu_core, to_dev  # noqa: E402


MODES = [1, 2, 3]


@pytest.fixture(scope="module", params=MODES, ids=["async", "bsp", "offline"])
def kc(request):
    with KCore(0, sync_mode=request.param) as k:
        yield k


def _csr(n, s, d):
    return oracle.build_csr(n, s, d)


@pytest.mark.parametrize("name", golden_io.names())
def test_golden(kc, name):
    n, s, d, want = golden_io.load(name)
    off, adj = _csr(n, s, d)
    assert_parity(kc, n, off, adj, want)


CLOSED = [gg.complete(1), gg.complete(2), gg.complete(60), gg.path(2), gg.path(1000),
          gg.star(5000), gg.cycle(3), gg.cycle(777), gg.complete_bipartite(7, 40),
          gg.grid2d(30, 41), gg.grid3d(9, 10, 11), gg.random_tree(5000, 3), gg.staircase(300)]


@pytest.mark.parametrize("i", range(len(CLOSED)))
def test_closed_forms(kc, i):
    n, s, d = CLOSED[i]
    off, adj = _csr(n, s, d)
    assert_parity(kc, n, off, adj)


def test_empty_graph(kc):
    o, a = to_dev(np.zeros(1, np.int64), np.zeros(0, np.int32))
    core, km = kc.decompose(o, a)
    assert core.numel() == 0 and int(km.cpu()[0]) == 0


def test_single_vertex_and_isolated(kc):
    for n in (1, 2, 1000):
        off = np.zeros(n + 1, np.int64)
        got, km = gpu_core(kc, off, np.zeros(0, np.int32))
        assert (got == 0).all() and km == 0


@pytest.mark.parametrize("seed", range(60))
def test_random_small(kc, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 400))
    n, s, d = gg.small_random(n, int(rng.integers(0, 6 * n)), 7000 + seed)
    off, adj = _csr(n, s, d)
    assert_parity(kc, n, off, adj)


@pytest.mark.parametrize("seed", range(8))
def test_random_rmat_small(kc, seed):
    s, d = gg.rmat(12, 8, seed=100 + seed, perm_seed=200 + seed)
    off, adj = _csr(1 << 12, s, d)
    assert_parity(kc, 1 << 12, off, adj)


def test_er10k(kc):
    n, s, d = gg.workload_er10k()
    off, adj = _csr(n, s, d)
    got = assert_parity(kc, n, off, adj)
    assert oracle.check(n, off, adj, got)[0] == 0


def test_union_of_shapes(kc):
    n, s, d = gg.disjoint_union(gg.complete(100), gg.path(3000), gg.staircase(150),
                                gg.grid2d(50, 50), gg.star(20000), gg.cycle(10))
    off, adj = _csr(n, s, d)
    assert_parity(kc, n, off, adj)


@pytest.mark.parametrize("opts", [
    dict(slice_arcs=16), dict(slice_arcs=128), dict(slice_arcs=4096), dict(local_queue=0),
    dict(local_queue=128),
    dict(ctas_per_sm=1), dict(min_ctas=1, vertices_per_cta=1 << 40), dict(vertices_per_cta=1),
])
@pytest.mark.parametrize("mode", MODES)
def test_tuning_modes(opts, mode):
    n, s, d = gg.disjoint_union((30000, *gg.rmat_n(30000, 300000, seed=5)), gg.staircase(120),
                                gg.path(2000), gg.star(3000))
    off, adj = _csr(n, s, d)
    want = oracle.bz(n, off, adj)
    with KCore(0, sync_mode=mode, **opts) as k:
        assert_parity(k, n, off, adj, want)


def test_star_hub(kc):
    n, s, d = gg.star(1_000_000)
    off, adj = _csr(n, s, d)
    got, km = gpu_core(kc, off, adj)
    assert (got == 1).all() and km == 1


def test_long_path(kc):
    n, s, d = gg.path(1_000_000)
    off, adj = _csr(n, s, d)
    got, km = gpu_core(kc, off, adj)
    assert (got == 1).all() and km == 1


def test_staircase_many_levels(kc):
    n, s, d = gg.staircase(2000)
    off, adj = _csr(n, s, d)
    got = assert_parity(kc, n, off, adj)
    assert got.max() == 2000
    st = kc.stats()
    assert st["kmax"] == 2000 and st["rounds"] >= 2000


def test_each_vertex_processed_once(kc):
    """Every vertex with arcs is processed exactly once (Theorem 1's proof):
    as global slices or from a warp-local queue."""
    n = 50000
    s, d = gg.rmat_n(n, 400000, seed=9)
    off, adj = _csr(n, s, d)
    assert_parity(kc, n, off, adj)
    st = kc.stats()
    deg = np.diff(off)
    sl = st["slice_arcs"]
    assert sl == (512 if st["sync_mode"] == 1 else 32)
    slices = int(np.sum((deg + sl - 1) // sl))
    # each vertex with arcs is taken once as a whole item (from the global or a
    # warp-local queue) and its list is split into ceil(deg / slice) slices
    assert st["items"] + st["local_items"] == slices


def test_host_entry_point(kc):
    n, s, d = gg.workload_er10k()
    off, adj = _csr(n, s, d)
    core, km = kc.decompose_host(off, adj)
    want = oracle.bz(n, off, adj)
    np.testing.assert_array_equal(core, want)
    assert km == want.max()


@pytest.mark.parametrize("mode", MODES)
def test_caller_workspace(mode):
    n = 20000
    s, d = gg.rmat_n(n, 100000, seed=3)
    off, adj = _csr(n, s, d)
    with KCore(0, sync_mode=mode) as k:
        ws = torch.empty(k.workspace_size(n, len(adj)), dtype=torch.uint8, device="cuda:0")
        k.set_workspace(ws)
        assert_parity(k, n, off, adj)
        small = torch.empty(1024, dtype=torch.uint8, device="cuda:0")
        k.set_workspace(small)
        o, a = to_dev(off, adj)
        with pytest.raises(KCoreError) as e:
            k.decompose(o, a)
        assert e.value.code == "OOM"


@pytest.mark.parametrize("mode,tail", [(1, None), (2, None), (3, None), (2, (0, 0)), (2, (1 << 30, 1 << 30))],
                         ids=["async", "bsp", "offline", "bsp-no-tail", "bsp-all-tail"])
def test_timeout_is_reported_and_context_survives(mode, tail):
    """A wait that can never be satisfied (CTA 0 withholds its completion
    token, its arrival at the first grid barrier, or -- in tail mode -- its
    first release of the parked CTAs) must end at the time limit with
    KCORE_ERR_TIMEOUT, and the same context must then decompose normally."""
    n = 5000
    s, d = gg.rmat_n(n, 40000, seed=1)
    off, adj = _csr(n, s, d)
    o, a = to_dev(off, adj)
    extra = {} if tail is None else dict(tail_items=tail[0], tail_entries=tail[1])
    with KCore(0, timeout_ms=200, test_stall=1, sync_mode=mode, **extra) as k:
        with pytest.raises(KCoreError) as e:
            k.decompose(o, a)
        assert e.value.code == "TIMEOUT"
        k.set_option("test_stall", 0)
        assert_parity(k, n, off, adj)


def test_malformed_offsets_rejected_on_device(kc):
    off = np.array([0, 2, 1, 3], np.int64)  # decreasing offsets
    adj = np.array([1, 2, 0], np.int32)
    o, a = to_dev(off, adj)
    with pytest.raises(KCoreError) as e:
        kc.decompose(o, a)
    assert e.value.code == "NOT_SIMPLE"


def test_out_of_range_neighbour_rejected(kc):
    off = np.array([0, 1, 2], np.int64)
    adj = np.array([1, 7], np.int32)  # 7 is not a vertex
    o, a = to_dev(off, adj)
    with pytest.raises(KCoreError) as e:
        kc.decompose(o, a)
    assert e.value.code == "NOT_SIMPLE"


def test_argument_errors(kc):
    o, a = to_dev(np.array([0, 1, 2], np.int64), np.array([1, 0], np.int32))
    L = kc._L
    assert L.kcore_decompose(kc._h, -1, 2, o.data_ptr(), a.data_ptr(), None, None, None) == 1
    assert L.kcore_decompose(kc._h, 2, 2, None, a.data_ptr(), None, None, None) == 1
    with pytest.raises(KCoreError):
        kc.set_option("slice_arcs", 1)


def test_bsp_counters_and_trace():
    """Bulk-synchronous schedule: one barrier per scan and per subround pass
    (plus the final scan that finds nothing left), one trace entry per
    non-empty level, the levels of the trace being exactly the distinct
    coreness values."""
    n = 60000
    s, d = gg.rmat_n(n, 500000, seed=21)
    off, adj = _csr(n, s, d)
    want = oracle.bz(n, off, adj)
    # (a batch-updated heavy subround takes two barriers: counted here without)
    with KCore(0, sync_mode=2, trace=1, batch_update=0) as k:
        assert_parity(k, n, off, adj, want)
        st = k.stats()
        tr = k.trace()
    assert st["sync_mode"] == 2
    assert st["passes"] > 0
    # a phase ends at a grid barrier, or at a CTA barrier in tail mode
    assert st["barriers"] + st["tail_phases"] - (st["rounds"] + st["passes"]) in (0, 1)
    levels = tr[:, 3].astype(np.int64)
    assert len(levels) == st["rounds"] - st["empty_rounds"]
    np.testing.assert_array_equal(levels, np.unique(want))
    assert int(tr[:, 13].sum()) == st["passes"]
    assert (tr[:, 2] >= tr[:, 1]).all() and (tr[:, 1] >= tr[:, 0]).all()


@pytest.mark.parametrize("batch_update", [0, 1])
def test_bsp_phase_trace(batch_update):
    """Trace mode 2: one record per grid barrier, in time order, levels
    non-decreasing; without the batch update the passes read every arc once
    (each vertex's list is traversed exactly once), and the scans' found
    counts sum to the vertices they took."""
    n = 60000
    s, d = gg.rmat_n(n, 500000, seed=22)
    off, adj = _csr(n, s, d)
    want = oracle.bz(n, off, adj)
    with KCore(0, sync_mode=2, trace=2, batch_update=batch_update) as k:
        assert_parity(k, n, off, adj, want)
        st = k.stats()
        tr = k.trace().astype(np.int64)
    assert len(tr) == st["barriers"] + st["tail_phases"]
    assert (np.diff(tr[:, 0]) >= 0).all()
    kinds = tr[:, 1]
    assert set(np.unique(kinds)) <= {0, 1, 2, 3, 4}
    # field 7 flags the phases CTA 0 ran alone; no counting or apply phase is among them
    assert int(tr[:, 7].sum()) == st["tail_phases"]
    assert not ((tr[:, 7] == 1) & ((kinds == 2) | (kinds == 3))).any()
    assert (np.diff(tr[:, 2]) >= 0).all()
    assert int(np.count_nonzero(kinds == 1)) + int(np.count_nonzero(kinds == 3)) == st["passes"]
    # a scan per visited level (two for an empty one), and perhaps a last
    # scan that finds nothing left
    assert int(np.count_nonzero((kinds == 0) | (kinds == 4))) - st["rounds"] in (0, 1)
    assert int(np.count_nonzero(kinds == 4)) == st["empty_rounds"]
    if batch_update == 0:
        assert int(tr[kinds == 1, 6].sum()) == len(adj)
    assert set(np.unique(tr[kinds == 1, 2])) <= set(np.unique(want).tolist())


@pytest.mark.parametrize("mode", MODES)
def test_isolated_only_and_single_level(mode):
    """Graphs whose vertices all share one coreness: isolated vertices only,
    a perfect matching, one clique."""
    with KCore(0, sync_mode=mode) as k:
        for n, s, d in [(1000, np.zeros(0, np.int32), np.zeros(0, np.int32)),
                        (2000, np.arange(0, 2000, 2, dtype=np.int32), np.arange(1, 2000, 2, dtype=np.int32)),
                        gg.complete(300)]:
            off, adj = _csr(n, s, d)
            assert_parity(k, n, off, adj)


@pytest.mark.parametrize("seed", range(6))
def test_offline_subrounds_are_algorithm_1s(seed):
    """Mode 3 applies each subround's decrements in one batch (Algorithm 2),
    so its subrounds are exactly those of Algorithm 1 with the sequential Peel
    (the oracle counts them), and its non-empty levels are the oracle's."""
    n = 4000 + 3000 * seed
    s, d = gg.rmat_n(n, 10 * n, seed=40 + seed)
    n2, s2, d2 = gg.disjoint_union((n, s, d), gg.staircase(60), gg.complete(30), gg.path(500),
                                   (20, np.zeros(0, np.int32), np.zeros(0, np.int32)))
    off, adj = _csr(n2, s2, d2)
    core, st = oracle.alg1(n2, off, adj)
    with KCore(0, sync_mode=3) as k:
        got = assert_parity(k, n2, off, adj, core)
        gs = k.stats()
    assert gs["sync_mode"] == 3
    assert gs["passes"] == st["subrounds"]
    assert gs["rounds"] - gs["empty_rounds"] == st["nonempty_rounds"]
    assert gs["local_items"] == 0


@pytest.mark.parametrize("W", [1, 2, 7, 16, 64, 100000])
def test_level_window(W):
    """Bucketing of the active list (mode 2, KCORE_OPT_LEVEL_WINDOW): the same
    coreness for every window size, on graphs with many levels, empty levels
    between them, isolated vertices and hubs."""
    n0 = 30000
    s, d = gg.rmat_n(n0, 300000, seed=5)
    n, s2, d2 = gg.disjoint_union((n0, s, d), gg.staircase(120), gg.path(2000), gg.star(3000),
                                  gg.complete(45), (17, np.zeros(0, np.int32), np.zeros(0, np.int32)))
    off, adj = _csr(n, s2, d2)
    want = oracle.bz(n, off, adj)
    with KCore(0, level_window=W, trace=1) as k:
        assert_parity(k, n, off, adj, want)
        st = k.stats()
        tr = k.trace()
        # every closed form and random graph of the earlier tests as well
        for i in range(len(CLOSED)):
            nn, ss, dd = CLOSED[i]
            o2, a2 = _csr(nn, ss, dd)
            assert_parity(k, nn, o2, a2)
    assert st["sync_mode"] == 2
    levels = tr[:, 3].astype(np.int64)
    np.testing.assert_array_equal(levels, np.unique(want))
    rebuilds = int(tr[:, 10].sum())
    assert rebuilds >= 1
    if W == 1:
        assert rebuilds >= len(levels) // 2  # a rebuild (almost) every level


@pytest.mark.parametrize("opts", [dict(), dict(precheck_items=0), dict(precheck_items=1 << 20)])
def test_batch_update_of_heavy_subrounds(opts):
    """KCORE_OPT_BATCH_UPDATE: heavy subrounds count decrements with
    reductions and apply them walking the active list; the coreness is the
    oracle's on graphs with dense cores, hubs, long paths and many levels,
    whether the other subrounds read d~ first or not."""
    n0 = 40000
    s, d = gg.rmat_n(n0, 600000, seed=8)
    n, s2, d2 = gg.disjoint_union((n0, s, d), gg.complete(200), gg.staircase(150), gg.star(5000),
                                  gg.path(3000), (9, np.zeros(0, np.int32), np.zeros(0, np.int32)))
    off, adj = _csr(n, s2, d2)
    want = oracle.bz(n, off, adj)
    with KCore(0, batch_update=1, **opts) as k:
        assert_parity(k, n, off, adj, want)
        for i in range(len(CLOSED)):
            nn, ss, dd = CLOSED[i]
            o2, a2 = _csr(nn, ss, dd)
            assert_parity(k, nn, o2, a2)
        for seed in range(4):
            nn = 20000
            ss, dd = gg.rmat_n(nn, 30 * nn, seed=70 + seed)
            o2, a2 = _csr(nn, ss, dd)
            assert_parity(k, nn, o2, a2)
