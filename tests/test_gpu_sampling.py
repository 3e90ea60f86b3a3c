"""The sampled peel (Sec. 4.1, Algorithms 4-5) and warp-aggregated decrements
(its alternative for hub contention) on the GPU, through the C ABI:
bit-exact coreness against Batagelj-Zaversnik on graphs with hubs, cliques
and long paths, over mu, thresholds and seeds; the coins are the oracle's
(Philox4x32-10 of the arc index), so on a star the GPU's heads and its
reruns (a missed level found by the recount test) equal the oracle's run by
run; every rerun still returns the exact coreness (Las Vegas)."""
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


def _run(k, off, adj, **opts):
    old = {name: k.get_option(name) for name in opts}
    for name, v in opts.items():
        k.set_option(name, v)
    try:
        o, a = to_dev(off, adj)
        core, km = k.decompose(o, a)
        return core.cpu().numpy(), int(km.item()), k.stats()
    finally:
        for name, v in old.items():
            k.set_option(name, v)


GRAPHS = {
    "star": lambda: gg.star(3000),
    "complete": lambda: gg.complete(150),
    "rmat12": lambda: (4096, *gg.rmat_n(4096, 60_000, seed=3)),
    "rmat16": lambda: (1 << 16, *gg.rmat_n(1 << 16, 1_000_000, seed=5)),
    "union": lambda: gg.disjoint_union(gg.complete(120), gg.star(900), gg.staircase(60), gg.complete(40),
                                       gg.path(3000), gg.cycle(500)),
    "knn_cliques": lambda: _knn_cliques(40_000),
}


def _knn_cliques(n):
    s1, d1 = gg.knn2d(n, 10, seed=3)
    s2, d2, _, _ = gg.planted_cliques(n, 8, 60, 400, seed=4)
    return n, np.concatenate([s1, s2]), np.concatenate([d1, d2])


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("mu,thr", [(8, 10), (60, 50), (0, -1)])
def test_sampled_peel_is_exact(kc, name, mu, thr):
    n, s, d = GRAPHS[name]()
    off, adj = oracle.build_csr(n, s, d)
    want = oracle.bz(n, off, adj)
    deg = np.diff(off)
    for seed in range(3):
        core, km, st = _run(kc, off, adj, sampling=1, sample_mu=mu, sample_threshold=thr, sample_seed=seed)
        np.testing.assert_array_equal(core, want)
        assert km == int(want.max())
        t = thr if thr >= 0 else 8 * (mu if mu > 0 else int(np.ceil(40 * np.log(max(n, 2)))))
        assert st["sample_vertices"] == int(np.count_nonzero(deg > t))
        assert st["sample_reruns"] in (0, 1)


def test_star_coins_and_reruns_match_the_oracle(kc):
    # all L leaves are peeled in level 1, each tossing its arc's coin for the
    # centre; the centre is recounted in level 1 only if mu heads came up,
    # otherwise the recount of level 2 finds the miss: same coins, same runs
    L, mu = 4000, 60
    n, s, d = gg.star(L)
    off, adj = oracle.build_csr(n, s, d)
    reruns = 0
    for seed in range(40):
        ok, _, ost = oracle.kcore_sampled(n, off, adj, mu, 100, seed)
        core, km, st = _run(kc, off, adj, sampling=1, sample_mu=mu, sample_threshold=100, sample_seed=seed)
        assert (core == 1).all() and km == 1
        assert st["sample_vertices"] == 1
        assert st["sample_heads"] == ost["heads"]
        assert st["sample_reruns"] == (0 if ok else 1)
        if not ok:
            assert st["sample_miss_round"] == ost["miss_round"] == 2
        reruns += st["sample_reruns"]
    assert 0 < reruns < 40


def test_sampled_without_final_check_is_exact(kc):
    n, s, d = GRAPHS["rmat16"]()
    off, adj = oracle.build_csr(n, s, d)
    want = oracle.bz(n, off, adj)
    for seed in range(3):
        core, _, st = _run(kc, off, adj, sampling=1, sample_mu=20, sample_threshold=30, sample_seed=seed,
                           sample_check=0)
        np.testing.assert_array_equal(core, want)
        assert st["sample_recounts"] >= st["sample_failed_validations"] > 0


def test_nothing_sampled_matches_default(kc):
    n, s, d = GRAPHS["union"]()
    off, adj = oracle.build_csr(n, s, d)
    core, _, st = _run(kc, off, adj, sampling=1, sample_threshold=int(np.diff(off).max()))
    np.testing.assert_array_equal(core, oracle.bz(n, off, adj))
    assert st["sample_vertices"] == 0 and st["sample_heads"] == 0 and st["sample_reruns"] == 0


def test_sampling_options_are_checked(kc):
    for name, bad in [("sampling", 2), ("sample_check", -1), ("sample_mu", -1), ("sample_mu", 1 << 25),
                      ("sample_threshold", -2)]:
        with pytest.raises(KCoreError):
            kc.set_option(name, bad)


def test_sampling_ignored_by_core_mask_and_other_modes(kc):
    n, s, d = GRAPHS["rmat12"]()
    off, adj = oracle.build_csr(n, s, d)
    want = oracle.bz(n, off, adj)
    for mode in (1, 3):
        core, _, st = _run(kc, off, adj, sampling=1, sync_mode=mode)
        np.testing.assert_array_equal(core, want)
        assert st["sample_vertices"] == 0
    core, _, _ = _run(kc, off, adj, sampling=1, level_window=8)
    np.testing.assert_array_equal(core, want)
    o, a = to_dev(off, adj)
    kc.set_option("sampling", 1)
    try:
        mask, size = kc.core_mask(o, a, 20)
    finally:
        kc.set_option("sampling", 0)
    wm, ws = oracle.kcore_mask(n, off, adj, 20)
    np.testing.assert_array_equal(mask.cpu().numpy(), wm)
    assert int(size.item()) == ws


@pytest.mark.slow
def test_sampled_rmat20_exact(kc):
    n = 1 << 20
    s, d = gg.rmat(20, 16, seed=1, perm_seed=2)
    off, adj = oracle.build_csr(n, s, d)
    want = oracle.bz(n, off, adj)
    core, km, st = _run(kc, off, adj, sampling=1)
    np.testing.assert_array_equal(core, want)
    assert st["sample_vertices"] > 0


@pytest.mark.parametrize("name", list(GRAPHS))
@pytest.mark.parametrize("batch_update", [0, 1])
def test_warp_combined_decrements_are_exact(kc, name, batch_update):
    # warp aggregation of decrements to one vertex: one atomic per group, the
    # crossing reported by the group whose interval holds the level
    n, s, d = GRAPHS[name]()
    off, adj = oracle.build_csr(n, s, d)
    core, km, st = _run(kc, off, adj, warp_combine=1, batch_update=batch_update)
    want = oracle.bz(n, off, adj)
    np.testing.assert_array_equal(core, want)
    assert km == int(want.max()) and st["sync_mode"] == 2
