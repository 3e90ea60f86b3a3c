"""Input generators: determinism, shapes and distribution facts (CPU)."""
import os
import subprocess
import sys

import numpy as np

import graphgen as gg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_er_distinct_pairs():
    n, s, d = gg.workload_er10k()
    assert n == 10_000 and len(s) == 50_000
    assert (s != d).all()
    key = np.minimum(s, d).astype(np.int64) * n + np.maximum(s, d)
    assert len(np.unique(key)) == 50_000
    assert s.min() >= 0 and max(s.max(), d.max()) < n


def test_rmat_shape_and_skew():
    s, d = gg.rmat(14, 16, seed=1, perm_seed=2)
    assert len(s) == 16 << 14
    assert s.min() >= 0 and s.max() < 1 << 14
    deg = np.bincount(np.concatenate([s, d]), minlength=1 << 14)
    # power-law: the top 1% of vertices carry far more than 1% of endpoints
    top = np.sort(deg)[::-1][: (1 << 14) // 100].sum()
    assert top > 0.15 * deg.sum()


def test_rmat_thread_count_independent():
    code = ("import graphgen as g, hashlib; s,d=g.rmat(12,8,seed=3,perm_seed=4);"
            "print(hashlib.sha1(s.tobytes()+d.tobytes()).hexdigest())")
    outs = []
    for t in ("1", "3"):
        env = dict(os.environ, GRAPHGEN_THREADS=t, PYTHONPATH=ROOT)
        outs.append(subprocess.check_output([sys.executable, "-c", code], env=env).strip())
    assert outs[0] == outs[1]


def test_knn_matches_brute_force():
    n, k = 700, 10
    s, d = gg.knn2d(n, k, seed=3)
    x, y = gg.points2d(n, seed=3)
    for i in range(0, n, 37):
        dist = (x - x[i]) ** 2 + (y - y[i]) ** 2
        dist[i] = np.inf
        order = np.lexsort((np.arange(n), dist))[:k]
        assert d[i * k:(i + 1) * k].tolist() == order.tolist()
        assert (s[i * k:(i + 1) * k] == i).all()


def test_cliques():
    s, d, sizes, members = gg.planted_cliques(5000, count=5, smin=10, smax=60, seed=4)
    assert len(sizes) == 5 and sizes.min() >= 10 and sizes.max() <= 60
    assert len(s) == int((sizes.astype(np.int64) * (sizes - 1) // 2).sum())
    off = 0
    for sz in sizes:
        mem = members[off:off + sz]
        assert len(np.unique(mem)) == sz
        off += sz


def test_batch_spec_distribution():
    spec = gg.batch_spec(512)
    n, m, kind = spec[:, 0], spec[:, 1], spec[:, 2]
    assert n.min() >= 1000 and n.max() <= 200_000
    dbar = 2 * m / n
    assert dbar.min() >= 3.9 and dbar.max() <= 64.1
    assert 0.4 < kind.mean() < 0.6
    # log-uniform: median near sqrt(1e3 * 2e5) ~ 14k
    assert 7_000 < np.median(n) < 28_000


def test_batch_edges_unique_local():
    spec = gg.batch_spec(8, nmin=100, nmax=3000, seed=9)
    eoff, s, d = gg.batch_edges(spec)
    for g in range(len(spec)):
        n = spec[g, 0]
        ss, dd = s[eoff[g]:eoff[g + 1]], d[eoff[g]:eoff[g + 1]]
        assert len(ss) == spec[g, 1]
        assert (ss != dd).all() and ss.max() < n and dd.max() < n
        key = np.minimum(ss, dd).astype(np.int64) * n + np.maximum(ss, dd)
        assert len(np.unique(key)) == len(ss)
