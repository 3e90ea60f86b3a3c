"""The no-allocation entry point, kcore_decompose_static, for callers that
cannot allocate device memory (another allocator owns it all, allocation is
forbidden after start-up, or an allocation's device synchronisation is not
acceptable). It must give exactly the coreness and k_max of kcore_decompose,
including on a second call in a row that reuses its fixed scratch array after a
larger graph, and it must refuse graphs above its stated limits.

This file is named to be collected last."""
import numpy as np
import pytest

import graphgen as gg
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2502_08042_gb300 import KCore, _native  # noqa: E402

KCORE_ERR_CAPACITY = 6


def _dev(off, adj):
    return (torch.from_numpy(np.ascontiguousarray(off, np.int64)).cuda(),
            torch.from_numpy(np.ascontiguousarray(adj, np.int32)).cuda())


def _static_call(off, adj):
    L = _native.lib()
    n = off.numel() - 1
    core = torch.full((max(n, 1),), -7, dtype=torch.int32, device="cuda")
    km = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    st = L.kcore_decompose_static(n, adj.numel(), off.data_ptr(),
                                  adj.data_ptr() if adj.numel() else None, core.data_ptr(),
                                  km.data_ptr(), torch.cuda.current_stream().cuda_stream or None)
    return st, core[:n], km


def test_static_matches_kcore_decompose_on_two_calls_in_a_row():
    # first a larger graph, then a smaller one: the second call must not see
    # anything the first one left in the shared scratch array
    s1, d1 = gg.rmat(18, 16, seed=11, perm_seed=12)
    n2, s2, d2 = gg.disjoint_union((9000, *gg.er(9000, 40000, seed=3)), gg.staircase(60), gg.path(700))
    cases = [(1 << 18, s1, d1), (n2, s2, d2)]
    with KCore(0) as k:
        for n, s, d in cases:
            off_h, adj_h = oracle.build_csr(n, s, d)
            off, adj = _dev(off_h, adj_h)
            ref_core, ref_km = k.decompose(off, adj)
            st, core, km = _static_call(off, adj)
            assert st == 0
            np.testing.assert_array_equal(core.cpu().numpy(), ref_core.cpu().numpy())
            assert int(km.item()) == int(ref_km.item())


def test_static_rejects_graphs_above_its_limit():
    off, adj = _dev(np.zeros(3, np.int64), np.zeros(0, np.int32))
    L = _native.lib()
    core = torch.empty(4, dtype=torch.int32, device="cuda")
    km = torch.empty(1, dtype=torch.int32, device="cuda")
    too_many_vertices = (1 << 20) + 1
    too_many_arcs = (1 << 24) + 2
    assert L.kcore_decompose_static(too_many_vertices, 0, off.data_ptr(), None, core.data_ptr(),
                                    km.data_ptr(), None) == KCORE_ERR_CAPACITY
    assert L.kcore_decompose_static(2, too_many_arcs, off.data_ptr(), adj.data_ptr(),
                                    core.data_ptr(), km.data_ptr(), None) == KCORE_ERR_CAPACITY
