"""Tail mode of the bulk-synchronous schedule (sync mode 2): subround passes
of at most KCORE_OPT_TAIL_ITEMS work items and scans of at most
KCORE_OPT_TAIL_ENTRIES active-list entries run on one CTA while the others
park. The coreness must equal the oracle's bit for bit at every threshold:
0 (never), 1 (only one-item passes and one-entry scans) and huge (the whole
peel on one CTA), on the closed forms, a staircase of 2,000 levels, R-MAT
graphs, and unions that switch between grid and tail phases many times."""
import numpy as np
import pytest

import graphgen as gg
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2502_08042_gb300 import KCore  # noqa: E402
from tests.gpu_util import assert_parity, to_dev  # noqa: E402
from tests.test_gpu_peel import CLOSED  # noqa: E402

HUGE = 1 << 30
THRESHOLDS = [(0, 0), (1, 1), (1, 0), (0, 1), (64, 4096), (256, 16384), (4096, 1 << 20), (HUGE, HUGE)]
IDS = ["off", "one", "items1", "entries1", "small", "default", "large", "all"]


@pytest.fixture(scope="module", params=THRESHOLDS, ids=IDS)
def kt(request):
    items, entries = request.param
    with KCore(0, sync_mode=2, tail_items=items, tail_entries=entries) as k:
        yield k


def test_closed_forms(kt):
    for n, s, d in CLOSED:
        off, adj = oracle.build_csr(n, s, d)
        assert_parity(kt, n, off, adj)


def test_staircase_2000(kt):
    n, s, d = gg.staircase(2000)
    off, adj = oracle.build_csr(n, s, d)
    got = assert_parity(kt, n, off, adj)
    assert got.max() == 2000


@pytest.mark.parametrize("seed", range(3))
def test_rmat(kt, seed):
    n = 1 << 15
    s, d = gg.rmat(15, 16, seed=30 + seed, perm_seed=31 + seed)
    off, adj = oracle.build_csr(n, s, d)
    assert_parity(kt, n, off, adj)


def test_union_switches_modes(kt):
    """A graph whose levels alternate between large and small phases: an
    R-MAT graph beside cliques, a staircase, stars, paths and isolated
    vertices."""
    s0, d0 = gg.rmat_n(40000, 500000, seed=12)
    n, s, d = gg.disjoint_union((40000, s0, d0), gg.staircase(300), gg.complete(150), gg.star(20000),
                                gg.path(5000), gg.grid2d(60, 70), (33, np.zeros(0, np.int32), np.zeros(0, np.int32)))
    off, adj = oracle.build_csr(n, s, d)
    assert_parity(kt, n, off, adj)


def test_counters():
    """With the thresholds at zero no phase runs in tail mode and every phase
    ends at a grid barrier; with huge thresholds every phase runs in tail mode
    after the parking (one episode, no grid barrier at all)."""
    n = 30000
    s, d = gg.rmat_n(n, 300000, seed=4)
    off, adj = oracle.build_csr(n, s, d)
    want = oracle.bz(n, off, adj)
    with KCore(0, sync_mode=2, tail_items=0, tail_entries=0) as k:
        assert_parity(k, n, off, adj, want)
        st0 = k.stats()
    assert st0["tail_phases"] == 0 and st0["tail_episodes"] == 0
    with KCore(0, sync_mode=2, tail_items=HUGE, tail_entries=HUGE) as k:
        assert_parity(k, n, off, adj, want)
        st1 = k.stats()
    assert st1["barriers"] == 0 and st1["tail_episodes"] == 1
    # one phase per scan (two for an empty level) and per pass, perhaps a last
    # scan that finds nothing left; no batch-updated pairs on one CTA
    assert st1["tail_phases"] - (st1["rounds"] + st1["passes"]) in (0, 1)
    # the same levels are visited either way
    assert st1["rounds"] == st0["rounds"] and st1["empty_rounds"] == st0["empty_rounds"]
    with KCore(0, sync_mode=2, tail_items=256, tail_entries=16384) as k:
        assert_parity(k, n, off, adj, want)
        st2 = k.stats()
    assert st2["tail_phases"] > 0 and st2["tail_episodes"] >= 1 and st2["barriers"] > 0
    # tail mode is off by default
    with KCore(0) as k:
        assert k.get_option("tail_items") == 0 and k.get_option("tail_entries") == 0


def test_phase_trace_marks_tail_phases():
    """Trace mode 2 records every phase; those CTA 0 ran alone carry the
    flag, and their ranges are within the thresholds."""
    n = 30000
    s, d = gg.rmat_n(n, 300000, seed=6)
    off, adj = oracle.build_csr(n, s, d)
    items, entries = 100, 3000
    with KCore(0, sync_mode=2, trace=2, tail_items=items, tail_entries=entries) as k:
        assert_parity(k, n, off, adj)
        st = k.stats()
        tr = k.trace().astype(np.int64)
    assert len(tr) == st["barriers"] + st["tail_phases"]
    solo = tr[:, 7] == 1
    assert int(solo.sum()) == st["tail_phases"] > 0
    kinds = tr[:, 1]
    assert (tr[solo & (kinds == 1), 3] <= items).all()
    assert (tr[solo & ((kinds == 0) | (kinds == 4)), 3] <= entries).all()
    assert (tr[~solo & (kinds == 1), 3] > items).all()


def test_options_switch_between_calls():
    """One handle, thresholds changed between calls: every result exact."""
    n, s, d = gg.disjoint_union((5000, *gg.er(5000, 30000, seed=2)), gg.staircase(120))
    off, adj = oracle.build_csr(n, s, d)
    want = oracle.bz(n, off, adj)
    o, a = to_dev(off, adj)
    with KCore(0, sync_mode=2) as k:
        for items, entries in [(HUGE, HUGE), (0, 0), (3, 100), (HUGE, 0), (0, HUGE)]:
            k.set_option("tail_items", items)
            k.set_option("tail_entries", entries)
            core, km = k.decompose(o, a)
            np.testing.assert_array_equal(core.cpu().numpy(), want)
            assert int(km.item()) == int(want.max())


def test_autotune_picks_a_schedule_and_keeps_exact_output():
    """kcore_autotune times its candidate schedules on the graph, leaves the
    fastest in the handle's options and the exact coreness in the outputs."""
    n0 = 30000
    s, d = gg.rmat_n(n0, 300000, seed=14)
    n, s2, d2 = gg.disjoint_union((n0, s, d), gg.staircase(200), gg.star(4000))
    off, adj = oracle.build_csr(n, s2, d2)
    want = oracle.bz(n, off, adj)
    o, a = to_dev(off, adj)
    with KCore(0) as k:
        k.set_option("trace", 1)
        core, km, t = k.autotune(o, a, repeats=2)
        np.testing.assert_array_equal(core.cpu().numpy(), want)
        assert int(km.item()) == int(want.max())
        assert t["candidates"] >= 8 and t["ms"] > 0
        assert k.get_option("sync_mode") == t["sync_mode"]
        assert k.get_option("tail_items") == t["tail_items"]
        assert k.get_option("tail_entries") == t["tail_entries"]
        assert k.get_option("precheck_items") == t["precheck_items"]
        assert k.get_option("trace") == 1  # restored
        k.set_option("trace", 0)
        core2, km2 = k.decompose(o, a)
        np.testing.assert_array_equal(core2.cpu().numpy(), want)


def test_autotune_rejects_bad_arguments():
    o, a = to_dev(np.array([0, 1, 2], np.int64), np.array([1, 0], np.int32))
    with KCore(0) as k:
        with pytest.raises(Exception):
            k.autotune(o, a, repeats=0)
