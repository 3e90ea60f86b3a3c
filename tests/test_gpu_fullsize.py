"""Parity at the full sizes of the benchmark workloads, in the launch
configuration bench.py times (a handle with default options): R-MAT scale 24
(16.8 M vertices, 268 M pairs drawn) and the 10-NN graph of 2^24 points with
64 planted cliques. The GPU-built CSR equals the oracle's bit for bit, and the
GPU coreness equals Batagelj-Zaversnik's on it and passes the certificate
check; the built CSR passes the GPU's simple-CSR check, and the kNN coreness
meets the workload's lower bounds (10 everywhere, s - 1 on a planted clique
of s vertices). Slow (generation and the single-core oracle take a minute or two)."""
import numpy as np
import pytest

import graphgen as gg
import oracle

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

from paper_2502_08042_gb300 import KCore  # noqa: E402


def _full_check(n, s, d):
    with KCore(0) as k:
        off_d, adj_d = k.build_csr(n, torch.from_numpy(s).cuda(), torch.from_numpy(d).cuda())
        k.validate_csr(off_d, adj_d)  # raises unless the built CSR is simple
        core_d, km_d = k.decompose(off_d, adj_d)
        st = k.stats()
        off, adj = off_d.cpu().numpy(), adj_d.cpu().numpy()
        core = core_d.cpu().numpy()
        kmax = int(km_d.item())
    del off_d, adj_d, core_d
    want_off, want_adj = oracle.build_csr(n, s, d)
    np.testing.assert_array_equal(off, want_off)
    np.testing.assert_array_equal(adj, want_adj)
    want = oracle.bz(n, off, adj)
    np.testing.assert_array_equal(core, want)
    assert kmax == int(want.max())
    assert oracle.check(n, off, adj, core) == (0, -1)
    return st, kmax, core


def test_rmat24_full_size():
    s, d = gg.rmat(24, 16, seed=1, perm_seed=2)
    st, kmax, _ = _full_check(1 << 24, s, d)
    assert st["sync_mode"] == 2 and kmax == 1622


def test_knn_cliques_full_size():
    n, s, d, sizes, members = gg.workload_knn_cliques(1 << 24, 10, 64)
    st, kmax, core = _full_check(n, s, d)
    assert st["sync_mode"] == 2 and kmax >= int(max(sizes)) - 1
    # every vertex has its 10 nearest points as neighbours, so the whole graph
    # is a 10-core; a planted clique of s vertices is an (s-1)-core
    assert int(core.min()) >= 10
    at = 0
    for sz in sizes.tolist():
        assert int(core[members[at:at + sz]].min()) >= sz - 1
        at += sz
