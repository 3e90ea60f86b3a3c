"""The simple-CSR check on the GPU (kcore_validate_csr), through the C ABI,
against the oracle's check_simple: every CSR kcore_build_csr or the oracle
builds passes; every planted defect is reported with its check code, vertex
and arc; malformed offsets are caught before any arc is read."""
import numpy as np
import pytest

import graphgen as gg
import oracle
from tests import csr_defects

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2502_08042_gb300 import KCore, KCoreError  # noqa: E402
from tests.gpu_util import to_dev  # noqa: E402


@pytest.fixture(scope="module")
def kc():
    with KCore(0) as k:
        yield k


def _validate(k, off, adj):
    """(code, vertex, arc); code 0 for a simple CSR."""
    o, a = to_dev(off, adj)
    try:
        k.validate_csr(o, a)
    except KCoreError as e:
        assert e.code == "NOT_SIMPLE", str(e)
        st = k.stats()
        assert st["invalid_check"] > 0
        return st["invalid_check"], st["invalid_vertex"], st["invalid_arc"]
    assert k.stats()["invalid_check"] == 0
    return 0, -1, -1


GRAPHS = {
    "er3000": lambda: (3000, *gg.er(3000, 12000, seed=5)),
    "rmat14": lambda: (1 << 14, *gg.rmat_n(1 << 14, 200_000, seed=6)),
    "star": lambda: gg.star(50_000),
    "grid": lambda: gg.grid2d(120, 90),
    "complete": lambda: gg.complete(300),
}


@pytest.mark.parametrize("name", list(GRAPHS))
def test_simple_graphs_pass(kc, name):
    n, s, d = GRAPHS[name]()
    off, adj = oracle.build_csr(n, s, d)
    assert oracle.check_simple(n, off, adj) == 0
    assert _validate(kc, off, adj) == (0, -1, -1)


def test_gpu_built_csr_passes(kc):
    n = 1 << 16
    s, d = gg.rmat_n(n, 600_000, seed=9)
    # duplicates, reversed pairs and self-loops, which the builder drops
    s = np.concatenate([s, d[:5000], s[:3000], np.arange(100, dtype=np.int32)])
    d = np.concatenate([d, s[:5000], d[:3000], np.arange(100, dtype=np.int32)])
    off, adj = kc.build_csr(n, torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda())
    kc.validate_csr(off, adj)
    assert kc.stats()["invalid_check"] == 0


@pytest.mark.parametrize("kind", csr_defects.KINDS)
@pytest.mark.parametrize("seed", range(3))
def test_planted_defect_is_reported_where_planted(kc, kind, seed):
    rng = np.random.default_rng(100 + seed)
    n = 5000
    s, d = gg.er(n, 30_000, seed=seed) if seed != 1 else gg.rmat_n(n, 40_000, seed=seed)
    off, adj = oracle.build_csr(n, s, d)
    o, a, code, v, arc = csr_defects.plant(n, off, adj, kind, rng)
    assert oracle.check_simple(n, o, a) == csr_defects.ORACLE_CODE[code]
    assert _validate(kc, o, a) == (code, v, arc)


def test_offsets_checked_before_arcs(kc):
    n = 2000
    off, adj = oracle.build_csr(n, *gg.er(n, 8000, seed=3))
    m = len(adj)
    # offsets[n] != m: an extra trailing arc that no list owns
    assert _validate(kc, off, np.append(adj, np.int32(0))) == (2, n, m)
    # offsets[0] != 0: vertices 0..v0 start at 1 (v0 has two or more arcs,
    # so every offset stays monotone)
    v0 = int(np.flatnonzero(np.diff(off) > 1)[0])
    o = off.copy()
    o[: v0 + 1] = 1
    assert _validate(kc, o, adj) == (2, 0, 1)
    # a decreasing offset inside [0, m]: vertex v's list ends before it starts
    o = off.copy()
    v = n // 2
    o[v] = o[v + 1] + 1
    assert o[v] <= m
    assert _validate(kc, o, adj) == (1, v, int(o[v]))
    # offsets beyond m: caught by pass 1, the arc pass never reads past adj
    o = off.copy()
    o[n - 1] = m + 5
    code, vv, _ = _validate(kc, o, adj)
    assert code == 1 and vv in (n - 2, n - 1)


def test_swapped_entries(kc):
    # an unsorted list also breaks the binary searches of its neighbours, so
    # either failure may come first; the check must report one of them
    n = 3000
    off, adj = oracle.build_csr(n, *gg.er(n, 15000, seed=11))
    deg = np.diff(off)
    v = int(np.flatnonzero(deg >= 4)[0])
    a = adj.copy()
    j = int(off[v]) + 1
    a[j], a[j + 1] = a[j + 1], a[j]
    assert oracle.check_simple(n, off, a) in (6, 7)
    code, _, _ = _validate(kc, off, a)
    assert code in (5, 6)


def test_empty_and_tiny(kc):
    assert _validate(kc, np.zeros(1, np.int64), np.zeros(0, np.int32)) == (0, -1, -1)   # n = 0
    assert _validate(kc, np.zeros(2, np.int64), np.zeros(0, np.int32)) == (0, -1, -1)   # one isolated vertex
    assert _validate(kc, np.zeros(1001, np.int64), np.zeros(0, np.int32)) == (0, -1, -1)
    # the single edge {0, 1}
    assert _validate(kc, np.array([0, 1, 2], np.int64), np.array([1, 0], np.int32)) == (0, -1, -1)
    # one arc 0->1 without its reverse
    assert _validate(kc, np.array([0, 1, 1], np.int64), np.array([1], np.int32)) == (6, 0, 0)
    # a self-loop on a one-vertex graph
    assert _validate(kc, np.array([0, 1], np.int64), np.array([0], np.int32)) == (4, 0, 0)


def test_check_then_decompose(kc):
    # a CSR that passes the check decomposes to the oracle's coreness
    n = 1 << 15
    off, adj = oracle.build_csr(n, *gg.rmat_n(n, 400_000, seed=21))
    o, a = to_dev(off, adj)
    kc.validate_csr(o, a)
    core, km = kc.decompose(o, a)
    np.testing.assert_array_equal(core.cpu().numpy(), oracle.bz(n, off, adj))
