"""Sync mode 4 of the single-graph peel: the whole graph on one CTA, or on one
thread-block cluster of 2, 4 or 8 CTAs (the batched peel's kernel on a batch of
one). Coreness and k_max must equal the oracle's bit for bit on the closed
forms, a 2,000-level staircase, R-MAT graphs and a union of shapes, also
through host buffers and a caller-supplied workspace; a malformed CSR is
reported; the k'-core query keeps its own schedule."""
import numpy as np
import pytest

import graphgen as gg
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2502_08042_gb300 import KCore, KCoreError  # noqa: E402
from tests.gpu_util import assert_parity, to_dev  # noqa: E402
from tests.test_gpu_peel import CLOSED  # noqa: E402


@pytest.fixture(scope="module", params=[0, 2, 4, 8], ids=["cta", "cl2", "cl4", "cl8"])
def k4(request):
    with KCore(0, sync_mode=4, batch_cluster=request.param) as k:
        yield k


def test_closed_forms(k4):
    for n, s, d in CLOSED:
        off, adj = oracle.build_csr(n, s, d)
        assert_parity(k4, n, off, adj)
    assert k4.stats()["sync_mode"] == 4


def test_staircase_2000(k4):
    n, s, d = gg.staircase(2000)
    off, adj = oracle.build_csr(n, s, d)
    assert assert_parity(k4, n, off, adj).max() == 2000


@pytest.mark.parametrize("scale", [12, 16])
def test_rmat(k4, scale):
    s, d = gg.rmat(scale, 16, seed=40 + scale, perm_seed=41 + scale)
    off, adj = oracle.build_csr(1 << scale, s, d)
    assert_parity(k4, 1 << scale, off, adj)


def test_union_of_shapes(k4):
    s0, d0 = gg.rmat_n(60000, 700000, seed=13)
    n, s, d = gg.disjoint_union((60000, s0, d0), gg.staircase(250), gg.complete(120), gg.star(30000),
                                gg.path(4000), (50, np.zeros(0, np.int32), np.zeros(0, np.int32)))
    off, adj = oracle.build_csr(n, s, d)
    assert_parity(k4, n, off, adj)


def test_empty_graph(k4):
    o, a = to_dev(np.zeros(1, np.int64), np.zeros(0, np.int32))
    core, km = k4.decompose(o, a)
    assert core.numel() == 0 and int(km.cpu()[0]) == 0


def test_host_buffers_and_own_workspace():
    n, s, d = gg.disjoint_union(gg.staircase(400), gg.grid2d(50, 50))
    off, adj = oracle.build_csr(n, s, d)
    want = oracle.bz(n, off, adj)
    with KCore(0, sync_mode=4) as k:
        core, km = k.decompose_host(off, adj)
        np.testing.assert_array_equal(core, want)
        assert int(km) == int(want.max())
    with KCore(0, sync_mode=4, batch_cluster=4) as k:
        ws = torch.empty(k.workspace_size(n, len(adj)), dtype=torch.uint8, device="cuda")
        k.set_workspace(ws)
        o, a = to_dev(off, adj)
        core, km = k.decompose(o, a)
        np.testing.assert_array_equal(core.cpu().numpy(), want)


def test_malformed_csr_is_reported():
    n, s, d = gg.complete(100)
    off, adj = oracle.build_csr(n, s, d)
    bad = off.copy()
    bad[10] = bad[11] + 3  # offsets run backwards at vertex 10
    with KCore(0, sync_mode=4, batch_cluster=2) as k:
        o, a = to_dev(bad, adj)
        with pytest.raises(KCoreError) as e:
            k.decompose(o, a)
        assert e.value.code == "NOT_SIMPLE"
        assert_parity(k, n, off, adj)  # the handle still works


def test_core_mask_keeps_its_schedule():
    n, s, d = gg.disjoint_union(gg.staircase(60), gg.complete(30))
    off, adj = oracle.build_csr(n, s, d)
    want = oracle.bz(n, off, adj)
    with KCore(0, sync_mode=4) as k:
        o, a = to_dev(off, adj)
        mask, size = k.core_mask(o, a, 25)
        np.testing.assert_array_equal(mask.cpu().numpy().astype(bool), want >= 25)
        assert int(size) == int((want >= 25).sum())
