"""The no-allocation entry point, kcore_decompose_static, for callers that
cannot allocate device memory (another allocator owns it all, allocation is
forbidden after start-up, or an allocation's device synchronisation is not
acceptable). Its coreness and k_max must equal the oracle's and those of
kcore_decompose, bit for bit, on two calls in a row that reuse its fixed
scratch array (a larger graph first), on the shapes with the most levels, hubs
and degenerate cases; once its first call has set it up, later calls must
leave the device's memory use unchanged; and it must refuse graphs above its
stated limits.

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


def _static_call(off, adj, core=None, km=None):
    L = _native.lib()
    n = off.numel() - 1
    if core is None:
        core = torch.full((max(n, 1),), -7, dtype=torch.int32, device="cuda")
    if km is None:
        km = torch.full((1,), -7, dtype=torch.int32, device="cuda")
    st = L.kcore_decompose_static(n, adj.numel(), off.data_ptr(),
                                  adj.data_ptr() if adj.numel() else None, core.data_ptr(),
                                  km.data_ptr(), torch.cuda.current_stream().cuda_stream or None)
    return st, core[:n], km


def _check(n, s, d, k):
    off_h, adj_h = oracle.build_csr(n, s, d)
    want = oracle.bz(n, off_h, adj_h)
    off, adj = _dev(off_h, adj_h)
    ref_core, ref_km = k.decompose(off, adj)
    st, core, km = _static_call(off, adj)
    assert st == 0
    got = core.cpu().numpy()
    np.testing.assert_array_equal(got, want)
    np.testing.assert_array_equal(got, ref_core.cpu().numpy())
    assert int(km.item()) == int(ref_km.item()) == (int(want.max()) if n else 0)


def test_static_matches_the_oracle_and_kcore_decompose_on_two_calls_in_a_row():
    # first a larger graph, then a smaller one: the second call must not see
    # anything the first one left in the shared scratch array
    s1, d1 = gg.rmat(18, 16, seed=11, perm_seed=12)
    n2, s2, d2 = gg.disjoint_union((9000, *gg.er(9000, 40000, seed=3)), gg.staircase(60), gg.path(700))
    with KCore(0) as k:
        _check(1 << 18, s1, d1, k)
        _check(n2, s2, d2, k)


@pytest.mark.parametrize("shape", ["staircase", "star", "isolated", "clique", "rmat20"])
def test_static_shapes(shape):
    if shape == "staircase":
        n, s, d = gg.staircase(1000)
    elif shape == "star":
        n, s, d = gg.star(200000)
    elif shape == "isolated":
        n, s, d = gg.disjoint_union((5000, np.zeros(0, np.int32), np.zeros(0, np.int32)), gg.complete(40))
    elif shape == "clique":
        n, s, d = gg.complete(1500)
    else:
        n = 1 << 20
        s, d = gg.rmat(20, 8, seed=5, perm_seed=6)
    with KCore(0) as k:
        _check(n, s, d, k)


def test_static_empty_and_edgeless():
    with KCore(0) as k:
        # n == 0: k_max 0, nothing else written
        off, adj = _dev(np.zeros(1, np.int64), np.zeros(0, np.int32))
        st, core, km = _static_call(off, adj)
        assert st == 0 and core.numel() == 0 and int(km.item()) == 0
        # m == 0 (adj passed as NULL): every vertex has coreness 0
        for n in (1, 3000):
            _check(n, np.zeros(0, np.int32), np.zeros(0, np.int32), k)


def test_static_calls_leave_device_memory_unchanged():
    """After the first call on the device (the one-time set-up), a call
    changes neither the driver's free-memory count nor what torch's caching
    allocator has reserved."""
    n, s, d = gg.disjoint_union((20000, *gg.rmat_n(20000, 200000, seed=8)), gg.staircase(80))
    off_h, adj_h = oracle.build_csr(n, s, d)
    want = oracle.bz(n, off_h, adj_h)
    off, adj = _dev(off_h, adj_h)
    core = torch.empty(n, dtype=torch.int32, device="cuda")
    km = torch.empty(1, dtype=torch.int32, device="cuda")
    assert _static_call(off, adj, core, km)[0] == 0  # the set-up call
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    reserved0 = torch.cuda.memory_reserved()
    for _ in range(2):
        core.fill_(-7)
        st, _, _ = _static_call(off, adj, core, km)
        assert st == 0
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0
        assert torch.cuda.memory_reserved() == reserved0
        np.testing.assert_array_equal(core.cpu().numpy(), want)
        assert int(km.item()) == int(want.max())


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
