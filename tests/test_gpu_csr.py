"""Parity of the GPU CSR build (through the C ABI) with the CPU oracle's
builder: offsets and adjacency bit for bit, on multigraph inputs with
duplicates, reversed pairs and self-loops, and on the workload generators."""
import numpy as np
import pytest

import graphgen as gg
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2502_08042_gb300 import KCore, KCoreError  # noqa: E402


@pytest.fixture(scope="module")
def kc():
    with KCore(0) as k:
        yield k


def gpu_csr(k, n, s, d):
    S = torch.from_numpy(np.ascontiguousarray(s, np.int32)).cuda()
    D = torch.from_numpy(np.ascontiguousarray(d, np.int32)).cuda()
    off, adj = k.build_csr(n, S, D)
    return off.cpu().numpy(), adj.cpu().numpy()


def check_same(k, n, s, d):
    want_off, want_adj = oracle.build_csr(n, s, d)
    off, adj = gpu_csr(k, n, s, d)
    np.testing.assert_array_equal(off, want_off)
    np.testing.assert_array_equal(adj, want_adj)
    return off, adj


@pytest.mark.parametrize("seed", range(40))
def test_small_multigraphs(kc, seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 300))
    n, s, d = gg.small_random(n, int(rng.integers(0, 3000)), 50 + seed)
    check_same(kc, n, s, d)


def test_er10k(kc):
    n, s, d = gg.workload_er10k()
    check_same(kc, n, s, d)


@pytest.mark.parametrize("scale", [10, 16, 18])
def test_rmat(kc, scale):
    s, d = gg.rmat(scale, 16, seed=1, perm_seed=2)
    check_same(kc, 1 << scale, s, d)


def test_knn_and_cliques(kc):
    n, s, d, sizes, members = gg.workload_knn_cliques(n=50_000, cliques=4, smin=20, smax=200)
    check_same(kc, n, s, d)


def test_several_tiles_and_ragged_tail(kc):
    # 2 * E keys = 3 tiles of 4096 plus a ragged remainder, ids up to 2^20
    rng = np.random.default_rng(3)
    E = 3 * 2048 + 777
    s = rng.integers(0, 1 << 20, E).astype(np.int32)
    d = rng.integers(0, 1 << 20, E).astype(np.int32)
    d[::5] = s[::5]  # self-loops
    s = np.concatenate([s, d[:100]])  # reversed duplicates
    d = np.concatenate([d, s[:100]])
    check_same(kc, 1 << 20, s, d)


def test_empty_and_loops_only(kc):
    off, adj = gpu_csr(kc, 5, np.zeros(0, np.int32), np.zeros(0, np.int32))
    assert (off == 0).all() and len(adj) == 0
    off, adj = gpu_csr(kc, 3, np.array([0, 1, 2], np.int32), np.array([0, 1, 2], np.int32))
    assert (off == 0).all() and len(adj) == 0
    off, adj = gpu_csr(kc, 1, np.array([0], np.int32), np.array([0], np.int32))
    assert (off == 0).all() and len(adj) == 0


def test_out_of_range_rejected(kc):
    S = torch.tensor([0, 1], dtype=torch.int32, device="cuda")
    D = torch.tensor([1, 9], dtype=torch.int32, device="cuda")
    with pytest.raises(KCoreError) as e:
        kc.build_csr(4, S, D)
    assert e.value.code == "INVALID"


def test_csr_then_peel_matches_oracle(kc):
    s, d = gg.rmat(17, 16, seed=7, perm_seed=8)
    n = 1 << 17
    S = torch.from_numpy(s).cuda()
    D = torch.from_numpy(d).cuda()
    off, adj = kc.build_csr(n, S, D)
    core, km = kc.decompose(off, adj)
    o2, a2 = oracle.build_csr(n, s, d)
    want = oracle.bz(n, o2, a2)
    np.testing.assert_array_equal(core.cpu().numpy(), want)


@pytest.mark.parametrize("shift", [1, 2, 3])
def test_edge_arrays_not_16_byte_aligned(kc, shift):
    """Edge arrays that start 4, 8 or 12 bytes past a 16-byte boundary (views
    into larger tensors): the first radix pass then reads them with 4-byte
    copies. Several whole 1,024-edge tiles and a ragged last one."""
    s, d = gg.rmat(14, 16, seed=3, perm_seed=4)
    n = 1 << 14
    S = torch.zeros(s.size + 8, dtype=torch.int32, device="cuda")
    D = torch.zeros(d.size + 8, dtype=torch.int32, device="cuda")
    S[shift:shift + s.size] = torch.from_numpy(s).cuda()
    D[4 - shift:4 - shift + d.size] = torch.from_numpy(d).cuda()
    Sv, Dv = S[shift:shift + s.size], D[4 - shift:4 - shift + d.size]
    assert Sv.data_ptr() % 16 != 0 or Dv.data_ptr() % 16 != 0
    off, adj = kc.build_csr(n, Sv, Dv)
    want_off, want_adj = oracle.build_csr(n, s, d)
    np.testing.assert_array_equal(off.cpu().numpy(), want_off)
    np.testing.assert_array_equal(adj.cpu().numpy(), want_adj)


@pytest.mark.parametrize("n", [256, 1 << 16])
def test_top_vertex_with_repeats_and_loops(kc, n):
    """n a power of two, so the top vertex n - 1 has every id bit set, like
    the sentinel that marks self-loops: many edges to it, each repeated and
    reversed, with self-loops on it and elsewhere, over several tiles."""
    rng = np.random.default_rng(n)
    top = n - 1
    x = rng.integers(0, n, 5000).astype(np.int32)
    s = np.concatenate([x, np.full(5000, top, np.int32), x[:2000], np.full(300, top, np.int32),
                        rng.integers(0, n, 4000).astype(np.int32)])
    d = np.concatenate([np.full(5000, top, np.int32), x, np.full(2000, top, np.int32),
                        np.full(300, top, np.int32), rng.integers(0, n, 4000).astype(np.int32)])
    perm = rng.permutation(s.size)
    check_same(kc, n, s[perm], d[perm])


def test_long_runs_of_one_repeated_edge(kc):
    """One edge repeated 9,000 times (its copies span several 2,048-key tiles
    and CTA chunks of both sorted sequences) among a random graph."""
    rng = np.random.default_rng(5)
    n = 3000
    s = np.concatenate([np.full(9000, 17, np.int32), rng.integers(0, n, 20000).astype(np.int32)])
    d = np.concatenate([np.full(9000, 2999, np.int32), rng.integers(0, n, 20000).astype(np.int32)])
    perm = rng.permutation(s.size)
    check_same(kc, n, s[perm], d[perm])
