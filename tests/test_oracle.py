"""Pins of the CPU oracle against facts that do not come from the oracle:
hand-derived fixtures, closed forms, brute force from the definition,
Theorem 1's exact work count, and certificate checks that must reject wrong
answers. All CPU-only."""
import numpy as np
import pytest

import graphgen as gg
import oracle
from tests import csr_defects, golden_io


def _csr(n, s, d):
    return oracle.build_csr(n, s, d)


def _all_three(n, s, d):
    off, adj = _csr(n, s, d)
    c_bz = oracle.bz(n, off, adj)
    c_a1, st = oracle.alg1(n, off, adj)
    return off, adj, c_bz, c_a1, st


# ----------------------------------------------------------------- fixtures
@pytest.mark.parametrize("name", golden_io.names())
def test_golden_fixture(name):
    n, s, d, want = golden_io.load(name)
    off, adj, c_bz, c_a1, _ = _all_three(n, s, d)
    np.testing.assert_array_equal(c_bz, want)
    np.testing.assert_array_equal(c_a1, want)
    assert oracle.check(n, off, adj, want) == (0, -1)
    assert oracle.brute_coreness(n, s, d) == want.tolist()


# ----------------------------------------------------------------- closed forms
CLOSED = [
    ("K1", gg.complete(1), lambda n: [0] * n),
    ("K2", gg.complete(2), lambda n: [1] * n),
    ("K7", gg.complete(7), lambda n: [6] * n),
    ("K40", gg.complete(40), lambda n: [39] * n),
    ("path2", gg.path(2), lambda n: [1] * n),
    ("path50", gg.path(50), lambda n: [1] * n),
    ("star1000", gg.star(1000), lambda n: [1] * n),
    ("cycle3", gg.cycle(3), lambda n: [2] * n),
    ("cycle101", gg.cycle(101), lambda n: [2] * n),
    ("K3_5", gg.complete_bipartite(3, 5), lambda n: [3] * n),
    ("K9_4", gg.complete_bipartite(9, 4), lambda n: [4] * n),
    ("grid2x2", gg.grid2d(2, 2), lambda n: [2] * n),
    ("grid7x13", gg.grid2d(7, 13), lambda n: [2] * n),
    ("grid1x9", gg.grid2d(1, 9), lambda n: [1] * n),
    ("cube2", gg.grid3d(2, 2, 2), lambda n: [3] * n),
    ("cube4x5x6", gg.grid3d(4, 5, 6), lambda n: [3] * n),
    ("tree300", gg.random_tree(300, 7), lambda n: [1] * n),
]


@pytest.mark.parametrize("name,g,f", CLOSED, ids=[c[0] for c in CLOSED])
def test_closed_forms(name, g, f):
    n, s, d = g
    off, adj, c_bz, c_a1, st = _all_three(n, s, d)
    want = np.array(f(n), np.int32)
    np.testing.assert_array_equal(c_bz, want)
    np.testing.assert_array_equal(c_a1, want)
    assert oracle.check(n, off, adj, want)[0] == 0


def test_isolated_vertices():
    n = 17
    off, adj, c_bz, c_a1, st = _all_three(n, np.empty(0, np.int32), np.empty(0, np.int32))
    assert (c_bz == 0).all() and (c_a1 == 0).all()
    assert st["rounds"] == 1 and st["kmax"] == 0


def test_empty_graph():
    off, adj, c_bz, c_a1, st = _all_three(0, np.empty(0, np.int32), np.empty(0, np.int32))
    assert len(c_bz) == 0 and len(c_a1) == 0 and st["rounds"] == 0


@pytest.mark.parametrize("K", [2, 3, 10, 57, 200])
def test_staircase(K):
    n, s, d = gg.staircase(K)
    off, adj, c_bz, c_a1, st = _all_three(n, s, d)
    want = np.array([K] * (K + 1) + list(range(1, K)), np.int32)
    np.testing.assert_array_equal(c_bz, want)
    np.testing.assert_array_equal(c_a1, want)
    assert st["kmax"] == K and st["nonempty_rounds"] == K


def test_disjoint_union_is_per_component():
    parts = [gg.complete(6), gg.cycle(9), gg.star(4), gg.grid3d(2, 3, 2), gg.staircase(8)]
    n, s, d = gg.disjoint_union(*parts)
    off, adj = _csr(n, s, d)
    c = oracle.bz(n, off, adj)
    base = 0
    for pn, ps, pd in parts:
        po, pa = _csr(pn, ps, pd)
        np.testing.assert_array_equal(c[base:base + pn], oracle.bz(pn, po, pa))
        base += pn


# ----------------------------------------------------------------- brute force
@pytest.mark.parametrize("seed", range(150))
def test_brute_force_small_random(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 28))
    m = int(rng.integers(0, 3 * n + 1))
    n, s, d = gg.small_random(n, m, seed)
    off, adj, c_bz, c_a1, st = _all_three(n, s, d)
    want = np.array(oracle.brute_coreness(n, s, d), np.int32)
    np.testing.assert_array_equal(c_bz, want)
    np.testing.assert_array_equal(c_a1, want)
    assert oracle.check(n, off, adj, c_bz)[0] == 0


@pytest.mark.parametrize("seed", range(20))
def test_brute_force_dense_random(seed):
    rng = np.random.default_rng(1000 + seed)
    n = int(rng.integers(5, 22))
    p = rng.random() * 0.8 + 0.1
    iu, ju = np.triu_indices(n, 1)
    keep = rng.random(len(iu)) < p
    s, d = iu[keep].astype(np.int32), ju[keep].astype(np.int32)
    off, adj, c_bz, c_a1, _ = _all_three(n, s, d)
    want = np.array(oracle.brute_coreness(n, s, d), np.int32)
    np.testing.assert_array_equal(c_bz, want)
    np.testing.assert_array_equal(c_a1, want)


# ----------------------------------------------------------------- Theorem 1
@pytest.mark.parametrize("seed", range(10))
def test_theorem1_work_count(seed):
    """Sum over rounds of |A_k| equals sum_v (1 + coreness(v)) (Theorem 1's
    proof), and each vertex enters exactly one frontier."""
    n, s, d = gg.small_random(60 + 20 * seed, 300 + 90 * seed, 500 + seed)
    off, adj, c_bz, c_a1, st = _all_three(n, s, d)
    assert st["sum_active"] == int(np.sum(1 + c_bz.astype(np.int64)))
    assert st["frontier_inserts"] == n
    assert st["rounds"] == int(c_bz.max()) + 1
    assert st["sum_active"] <= n + len(adj)


def test_theorem1_on_er10k():
    n, s, d = gg.workload_er10k()
    off, adj, c_bz, c_a1, st = _all_three(n, s, d)
    np.testing.assert_array_equal(c_bz, c_a1)
    assert st["sum_active"] == int(np.sum(1 + c_bz.astype(np.int64)))
    assert st["frontier_inserts"] == n


# ----------------------------------------------------------------- certificate
def test_check_rejects_k4_all_two():
    """K4 with every value 2 passes (i) and (ii); only (iii) rejects it."""
    n, s, d = gg.complete(4)
    off, adj = _csr(n, s, d)
    code, bad = oracle.check(n, off, adj, np.full(4, 2, np.int32))
    assert code == 3 and bad >= 0


@pytest.mark.parametrize("seed", range(30))
def test_check_rejects_off_by_one(seed):
    rng = np.random.default_rng(seed)
    n, s, d = gg.small_random(40, 160, 900 + seed)
    off, adj = _csr(n, s, d)
    c = oracle.bz(n, off, adj)
    assert oracle.check(n, off, adj, c)[0] == 0
    for delta in (1, -1):
        bad = c.copy()
        v = int(rng.integers(0, n))
        if bad[v] + delta < 0:
            continue
        bad[v] += delta
        assert oracle.check(n, off, adj, bad)[0] != 0


def test_check_rejects_shifted_vector():
    n, s, d = gg.workload_er10k()
    off, adj = _csr(n, s, d)
    c = oracle.bz(n, off, adj)
    assert oracle.check(n, off, adj, c)[0] == 0
    assert oracle.check(n, off, adj, c + 1)[0] != 0
    assert oracle.check(n, off, adj, np.maximum(c - 1, 0))[0] != 0


# ----------------------------------------------------------------- CSR builder
@pytest.mark.parametrize("seed", range(40))
def test_build_csr_matches_set_definition(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 50))
    n, s, d = gg.small_random(n, int(rng.integers(0, 200)), seed)
    off, adj = _csr(n, s, d)
    nb = [set() for _ in range(n)]
    for a, b in zip(s.tolist(), d.tolist()):
        if a != b:
            nb[a].add(b)
            nb[b].add(a)
    assert off[0] == 0 and off[-1] == len(adj)
    for v in range(n):
        assert adj[off[v]:off[v + 1]].tolist() == sorted(nb[v])
    assert oracle.check_simple(n, off, adj) == 0


def test_check_simple_rejects_bad_csr():
    n, s, d = gg.cycle(6)
    off, adj = _csr(n, s, d)
    assert oracle.check_simple(n, off, adj) == 0
    a2 = adj.copy()
    a2[0] = 3  # 0 -> 3 has no reverse arc, and list order breaks
    assert oracle.check_simple(n, off, a2) != 0
    a3 = adj.copy()
    a3[off[2]] = 2  # self-loop
    assert oracle.check_simple(n, off, a3) != 0


@pytest.mark.parametrize("kind", csr_defects.KINDS)
def test_check_simple_finds_each_planted_defect(kind):
    # each planted defect is the only failure, so the oracle's first failed
    # check is the one planted
    rng = np.random.default_rng(7)
    for seed in range(4):
        n = 400
        s, d = gg.er(n, 1600, seed=seed) if seed % 2 == 0 else gg.rmat_n(n, 3000, seed=seed)
        off, adj = oracle.build_csr(n, s, d)
        o, a, code, v, arc = csr_defects.plant(n, off, adj, kind, rng)
        assert oracle.check_simple(n, o, a) == csr_defects.ORACLE_CODE[code]


def test_build_csr_rejects_out_of_range():
    with pytest.raises(ValueError):
        oracle.build_csr(3, np.array([0, 5], np.int32), np.array([1, 1], np.int32))


# ----------------------------------------------------------------- batch helper
def test_bz_batch_matches_union():
    spec = gg.batch_spec(6, nmin=50, nmax=400, seed=11)
    eoff, s, d = gg.batch_edges(spec)
    gv = np.zeros(len(spec) + 1, np.int64)
    np.cumsum(spec[:, 0], out=gv[1:])
    # union CSR with global ids
    gs = np.concatenate([s[eoff[g]:eoff[g + 1]].astype(np.int64) + gv[g] for g in range(len(spec))])
    gd = np.concatenate([d[eoff[g]:eoff[g + 1]].astype(np.int64) + gv[g] for g in range(len(spec))])
    N = int(gv[-1])
    off, adj = oracle.build_csr(N, gs.astype(np.int32), gd.astype(np.int32))
    want = oracle.bz(N, off, adj)
    # segmented CSR: same offsets, graph-local ids
    gid = np.repeat(np.arange(len(spec)), np.diff(gv))
    src_of_arc = np.repeat(np.arange(N), np.diff(off))
    local = adj - gv[gid[src_of_arc]]
    core, km = oracle.bz_batch(gv, off, local.astype(np.int32))
    np.testing.assert_array_equal(core, want)
    for g in range(len(spec)):
        assert km[g] == want[gv[g]:gv[g + 1]].max()


# ----------------------------------------------------------------- k'-core (App. B)
def _nbrs(n, off, adj):
    return [set(adj[off[v]:off[v + 1]].tolist()) for v in range(n)]


def _subset_union_core(n, nbrs, kp):
    """The k'-core from the definition by enumeration: the union of every
    vertex set whose induced subgraph has minimum degree >= kp (that union is
    itself such a set, the largest one)."""
    members = set()
    for bits in range(1, 1 << n):
        S = [v for v in range(n) if bits >> v & 1]
        Sset = set(S)
        if all(len(nbrs[v] & Sset) >= kp for v in S):
            members |= Sset
    return members


@pytest.mark.parametrize("seed", range(40))
def test_kcore_mask_matches_subset_enumeration(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 10))
    n, s, d = gg.small_random(n, int(rng.integers(0, 3 * n + 1)), seed=seed)
    off, adj = _csr(n, s, d)
    nb = _nbrs(n, off, adj)
    for kp in range(0, n + 1):
        mask, size = oracle.kcore_mask(n, off, adj, kp)
        want = _subset_union_core(n, nb, kp) if kp > 0 else set(range(n))
        assert set(np.flatnonzero(mask).tolist()) == want, (seed, kp)
        assert size == len(want)


@pytest.mark.parametrize("seed", range(30))
def test_kcore_mask_matches_definition_and_coreness(seed):
    """Against the pure-Python deletion of the definition (brute.py) and
    against Batagelj-Zaversnik coreness: v is in the k'-core iff coreness >= k'."""
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(5, 60))
    n, s, d = gg.small_random(n, int(rng.integers(n, 6 * n)), seed=100 + seed)
    off, adj = _csr(n, s, d)
    core = oracle.bz(n, off, adj)
    nb = _nbrs(n, off, adj)
    for kp in range(0, int(core.max()) + 3):
        mask, size = oracle.kcore_mask(n, off, adj, kp)
        np.testing.assert_array_equal(mask, (core >= kp).astype(np.int32))
        assert set(np.flatnonzero(mask).tolist()) == oracle.brute.k_core_members(n, nb, kp)
        assert size == int(mask.sum())


@pytest.mark.parametrize("name,g,kp,inside", [
    ("K12 k'=11", gg.complete(12), 11, True), ("K12 k'=12", gg.complete(12), 12, False),
    ("C30 k'=2", gg.cycle(30), 2, True), ("C30 k'=3", gg.cycle(30), 3, False),
    ("P50 k'=1", gg.path(50), 1, True), ("P50 k'=2", gg.path(50), 2, False),
    ("star k'=1", gg.star(40), 1, True), ("star k'=2", gg.star(40), 2, False),
    ("grid k'=2", gg.grid2d(9, 7), 2, True), ("grid k'=3", gg.grid2d(9, 7), 3, False),
    ("K5,8 k'=5", gg.complete_bipartite(5, 8), 5, True), ("K5,8 k'=6", gg.complete_bipartite(5, 8), 6, False),
], ids=lambda x: x if isinstance(x, str) else "")
def test_kcore_mask_closed_forms(name, g, kp, inside):
    """Closed forms: every vertex is in the k'-core or none is."""
    n, s, d = g
    off, adj = _csr(n, s, d)
    mask, size = oracle.kcore_mask(n, off, adj, kp)
    assert (mask == (1 if inside else 0)).all() and size == (n if inside else 0)


def test_kcore_mask_staircase_levels():
    """The staircase with K levels: its k'-core holds exactly the vertices of
    coreness >= k', and every member keeps >= k' neighbours inside it."""
    n, s, d = gg.staircase(40)
    off, adj = _csr(n, s, d)
    core = oracle.bz(n, off, adj)
    for kp in (1, 7, 20, 39, 40, 41):
        mask, size = oracle.kcore_mask(n, off, adj, kp)
        np.testing.assert_array_equal(mask, (core >= kp).astype(np.int32))
        inside = np.flatnonzero(mask)
        for v in inside:
            assert mask[adj[off[v]:off[v + 1]]].sum() >= kp


# ------------------------------------------------ sampling (Sec. 4.1, Algs. 4-5)
def test_philox_known_answers():
    # Philox4x32-10 known-answer vectors published with the generator
    # (Salmon et al., SC 2011; the Random123 known-answer tests)
    assert oracle.philox4x32_10((0, 0, 0, 0), (0, 0)) == (0x6627E8D5, 0xE169C58D, 0xBC57AC4C, 0x9B00DBD8)
    f = 0xFFFFFFFF
    assert oracle.philox4x32_10((f, f, f, f), (f, f)) == (0x408F276D, 0x41C83B0E, 0xA20BC7C6, 0x6D5451FD)
    assert oracle.philox4x32_10((0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344), (0xA4093822, 0x299F31D0)) \
        == (0xD16CFE09, 0x94FDCCEB, 0x5001E420, 0x24126EA1)


def _sampling_graphs():
    yield "star", gg.star(3000)
    yield "complete", gg.complete(150)
    yield "rmat", (4096, *gg.rmat_n(4096, 60_000, seed=3))
    yield "cliques", gg.disjoint_union(gg.complete(120), gg.star(900), gg.staircase(60), gg.complete(40))
    n = 20_000
    s1, d1 = gg.knn2d(n, 10, seed=3)
    s2, d2, _, _ = gg.planted_cliques(n, 6, 60, 300, seed=4)
    yield "knn+cliques", (n, np.concatenate([s1, s2]), np.concatenate([d1, d2]))


@pytest.mark.parametrize("name,g", list(_sampling_graphs()), ids=lambda x: x if isinstance(x, str) else "")
def test_sampled_peel_is_exact_or_reports_a_true_miss(name, g):
    # Values never fall below coreness (each is set when at most k untraversed
    # neighbours remain), so the recovery check can only fire on a vertex that
    # really missed an earlier round; without a report the result is exact
    n, s, d = g
    off, adj = oracle.build_csr(n, s, d)
    want = oracle.bz(n, off, adj)
    deg = np.diff(off)
    oks = 0
    for mu, thr in [(8, 10), (40, 30), (200, 50)]:
        for seed in range(6):
            ok, core, st = oracle.kcore_sampled(n, off, adj, mu, thr, seed)
            assert st["sampled_at_start"] == int(np.count_nonzero(deg > thr))
            if ok:
                oks += 1
                np.testing.assert_array_equal(core, want)
                assert st["miss_round"] == -1
            else:
                v = st["miss_vertex"]
                assert 0 <= v < n and want[v] < st["miss_round"]
    assert oks > 0


def test_sampled_peel_without_samples_is_algorithm_1():
    n, s, d = gg.disjoint_union(gg.complete(30), gg.staircase(25), gg.grid2d(9, 7))
    off, adj = oracle.build_csr(n, s, d)
    ok, core, st = oracle.kcore_sampled(n, off, adj, 50, int(np.diff(off).max()), 1)
    _, st1 = oracle.alg1(n, off, adj)
    assert ok and st["sampled_at_start"] == 0 and st["heads"] == 0 and st["recounts"] == 0
    np.testing.assert_array_equal(core, oracle.bz(n, off, adj))
    assert st["rounds"] == st1["rounds"]


def test_sampled_peel_complete_graph_never_misses():
    # K_n: every vertex sampled; Error(v, k) fails once 10 k >= n - 1, the
    # recount finds n - 1 untraversed neighbours, and the peel is exact
    n, s, d = gg.complete(200)
    off, adj = oracle.build_csr(n, s, d)
    for seed in range(5):
        ok, core, st = oracle.kcore_sampled(n, off, adj, 30, 10, seed)
        assert ok and (core == n - 1).all()
        assert st["sampled_at_start"] == n and st["failed_validations"] >= n


def test_sampling_coin_rate_and_counting_bag():
    # Star with L leaves, centre sampled: the leaves are peeled in round 1,
    # giving the centre L coins of probability p = floor(2^32 mu / ((1 - r) L)) / 2^32
    # (r = 1/10). The centre is recounted in round 1 only through the counting
    # bag (mu heads); otherwise it misses round 1 and the recovery check fires.
    scipy_stats = pytest.importorskip("scipy.stats")
    L, mu = 4000, 60
    n, s, d = gg.star(L)
    off, adj = oracle.build_csr(n, s, d)
    p = (10 * mu * 2**32 // (9 * L)) / 2**32
    heads, misses, trials = [], 0, 300
    for seed in range(trials):
        ok, core, st = oracle.kcore_sampled(n, off, adj, mu, 100, seed)
        heads.append(st["heads"])
        if ok:
            assert core[0] == 1 and (core == 1).all()
        else:
            misses += 1
            assert st["miss_vertex"] == 0
    mean, sd = L * p, np.sqrt(L * p * (1 - p))
    assert abs(np.mean(heads) - mean) < 5 * sd / np.sqrt(trials)
    q = scipy_stats.binom.cdf(mu - 1, L, p)  # P(fewer than mu heads)
    assert abs(misses - trials * q) < 5 * np.sqrt(trials * q * (1 - q)) + 1
