"""Parity of the k'-core query (App. B) on the GPU, through the C ABI, with the
oracle's repeated deletion: bit-exact membership and size for closed forms,
random graphs, the ER n=10,000 workload and R-MAT graphs, over thresholds
from 0 to beyond k_max."""
import numpy as np
import pytest

import graphgen as gg
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2502_08042_gb300 import KCore, KCoreError  # noqa: E402
from tests.gpu_util import to_dev  # noqa: E402


@pytest.fixture(scope="module")
def kc():
    with KCore(0) as k:
        yield k


def _check(k, n, off, adj, kprime):
    want, wsize = oracle.kcore_mask(n, off, adj, kprime)
    o, a = to_dev(off, adj)
    mask, size = k.core_mask(o, a, kprime)
    got = mask.cpu().numpy()
    np.testing.assert_array_equal(got, want)
    assert int(size.item()) == wsize
    return got


@pytest.mark.parametrize("g,kps", [
    (gg.complete(60), [0, 1, 58, 59, 60]),
    (gg.cycle(1000), [1, 2, 3]),
    (gg.path(5000), [1, 2]),
    (gg.star(20000), [1, 2]),
    (gg.grid2d(100, 70), [2, 3]),
    (gg.complete_bipartite(40, 90), [39, 40, 41]),
    (gg.staircase(300), [1, 50, 150, 299, 300, 301]),
])
def test_core_mask_closed_forms(kc, g, kps):
    n, s, d = g
    off, adj = oracle.build_csr(n, s, d)
    for kp in kps:
        _check(kc, n, off, adj, kp)


@pytest.mark.parametrize("seed", range(12))
def test_core_mask_random(kc, seed):
    n = 3000 + 1000 * seed
    s, d = gg.rmat_n(n, 12 * n, seed=seed)
    off, adj = oracle.build_csr(n, s, d)
    core = oracle.bz(n, off, adj)
    kmax = int(core.max())
    for kp in sorted({0, 1, 2, kmax // 3, kmax // 2, kmax, kmax + 1, 10 * kmax + 5}):
        _check(kc, n, off, adj, kp)


def test_core_mask_er10k_and_union(kc):
    n, s, d = gg.workload_er10k()
    off, adj = oracle.build_csr(n, s, d)
    for kp in range(0, 12):
        _check(kc, n, off, adj, kp)
    n, s, d = gg.disjoint_union(gg.complete(100), gg.path(3000), gg.staircase(150), gg.star(20000))
    off, adj = oracle.build_csr(n, s, d)
    for kp in (1, 2, 75, 99, 100, 149, 150, 151):
        _check(kc, n, off, adj, kp)


def test_core_mask_rmat_large(kc):
    """R-MAT scale 18 at the thresholds of the coreness distribution's
    quartiles: the query agrees with coreness >= k'."""
    s, d = gg.rmat(18, 16, seed=3, perm_seed=4)
    n = 1 << 18
    off, adj = oracle.build_csr(n, s, d)
    core = oracle.bz(n, off, adj)
    o, a = to_dev(off, adj)
    for q in (0.25, 0.5, 0.9, 0.999):
        kp = int(np.quantile(core, q))
        mask, size = kc.core_mask(o, a, kp)
        np.testing.assert_array_equal(mask.cpu().numpy(), (core >= kp).astype(np.int32))
        assert int(size.item()) == int((core >= kp).sum())


@pytest.mark.parametrize("opts", [dict(slice_arcs=16), dict(slice_arcs=1024), dict(local_queue=0),
                                  dict(sync_mode=1), dict(min_ctas=1, vertices_per_cta=1 << 40)])
def test_core_mask_options(opts):
    """Tuning options change the launch, not the answer (sync mode 1 does not
    apply: the query always runs the bulk-synchronous kernel)."""
    n = 20000
    s, d = gg.rmat_n(n, 200000, seed=11)
    off, adj = oracle.build_csr(n, s, d)
    with KCore(0, **opts) as k:
        for kp in (3, 17, 40):
            _check(k, n, off, adj, kp)


def test_core_mask_empty_and_errors(kc):
    o = torch.zeros(1, dtype=torch.int64, device="cuda:0")
    a = torch.zeros(0, dtype=torch.int32, device="cuda:0")
    mask, size = kc.core_mask(o, a, 3)
    assert mask.numel() == 0 and int(size.item()) == 0
    L = kc._L
    o2, a2 = to_dev(np.array([0, 1, 2], np.int64), np.array([1, 0], np.int32))
    assert L.kcore_core_mask(kc._h, 2, 2, o2.data_ptr(), a2.data_ptr(), 1, None, None, None) == 1
    assert L.kcore_core_mask(kc._h, -1, 0, None, None, 1, None, None, None) == 1
    # an id outside [0, n) on a list that is read is reported, as for the
    # decomposition: with k' = 2, vertices 0 and 2 are removed while vertex 1
    # is still kept, so their lists are read (vertex 2's holds the bad id)
    o3, a3 = to_dev(np.array([0, 1, 3, 4], np.int64), np.array([1, 0, 2, 7], np.int32))
    with pytest.raises(KCoreError) as e:
        kc.core_mask(o3, a3, 2)
    assert e.value.code == "NOT_SIMPLE"
