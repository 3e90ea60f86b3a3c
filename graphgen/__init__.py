"""Seeded synthetic graph generators shared by the tests, the benchmark and the
oracle's checks.

Every generator returns a raw edge list ``(src, dst)`` of int32 numpy arrays
(COO pairs). Nothing here builds a CSR, symmetrises, deduplicates or peels:
those steps belong to the CSR builders and the decomposition under test. The
heavy generators (R-MAT, kNN, batches) are C in ``graphgen.c``; the small
closed-form families are plain numpy below.

Workload classes follow the paper's evaluation set-up (Sec. 6.1): power-law
graphs (R-MAT stands in for the social/web graphs and the Barabasi-Albert HPL
graph), kNN graphs (a 2-D uniform point cloud stands in for GeoLife/Cosmo),
grids/cubes and the staircase graph (HCNS) with one vertex per coreness value.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libgraphgen.so")
_lock = threading.Lock()
_lib = None

# R-MAT quadrant probabilities used throughout (Graph500 values).
RMAT_ABC = (0.57, 0.19, 0.19)


def build(force: bool = False) -> str:
    """Compiles graphgen.c with the host gcc into _build/libgraphgen.so."""
    src = os.path.join(_HERE, "graphgen.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O3", "-std=gnu11", "-fPIC", "-shared", "-pthread",
                           "-o", tmp, src, "-lm"])
    os.replace(tmp, _SO)
    return _SO


def _L():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, u64, i32, dbl, p = (ctypes.c_int64, ctypes.c_uint64, ctypes.c_int,
                                     ctypes.c_double, ctypes.c_void_p)
            lib.gg_er.argtypes = [i64, i64, u64, p, p]
            lib.gg_rmat.argtypes = [i32, i64, dbl, dbl, dbl, u64, u64, i32, p, p]
            lib.gg_rmat_n.argtypes = [i64, i64, dbl, dbl, dbl, u64, p, p]
            lib.gg_knn2d.argtypes = [i64, i32, u64, p, p]
            lib.gg_points2d.argtypes = [i64, u64, p, p]
            lib.gg_cliques.argtypes = [i64, i32, i32, i32, u64, p, p, p, p]
            lib.gg_permutation.argtypes = [i64, u64, p]
            lib.gg_batch_spec.argtypes = [i64, i64, i64, dbl, dbl, u64, p]
            lib.gg_batch_edges.argtypes = [i64, p, p, dbl, dbl, dbl, p, p]
            for f in ("gg_er", "gg_rmat", "gg_rmat_n", "gg_knn2d", "gg_points2d", "gg_cliques",
                      "gg_permutation", "gg_batch_spec", "gg_batch_edges"):
                getattr(lib, f).restype = ctypes.c_int
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


def _check(rc: int, what: str) -> None:
    if rc != 0:
        raise RuntimeError(f"graphgen: {what} failed with code {rc}")


# --------------------------------------------------------------------------- generators
def er(n: int, m: int, seed: int = 1):
    """G(n, m): m distinct unordered non-loop pairs, uniform without replacement."""
    src = np.empty(m, np.int32)
    dst = np.empty(m, np.int32)
    _check(_L().gg_er(n, m, seed, _ptr(src), _ptr(dst)), "er")
    return src, dst


def rmat(scale: int, edge_factor: int = 16, seed: int = 1, perm_seed: int = 2,
         abc=RMAT_ABC, permute: bool = True, edges: int | None = None):
    """R-MAT edge list: edge_factor * 2^scale directed draws (duplicates and
    self-loops kept), ids randomly permuted with perm_seed."""
    e = edge_factor * (1 << scale) if edges is None else edges
    src = np.empty(e, np.int32)
    dst = np.empty(e, np.int32)
    a, b, c = abc
    _check(_L().gg_rmat(scale, e, a, b, c, seed, perm_seed, int(permute), _ptr(src), _ptr(dst)),
           "rmat")
    return src, dst


def rmat_n(n: int, m: int, seed: int, abc=RMAT_ABC):
    """R-MAT on exactly n vertices with m distinct undirected non-loop edges."""
    src = np.empty(m, np.int32)
    dst = np.empty(m, np.int32)
    a, b, c = abc
    _check(_L().gg_rmat_n(n, m, a, b, c, seed, _ptr(src), _ptr(dst)), "rmat_n")
    return src, dst


def points2d(n: int, seed: int):
    x = np.empty(n, np.float64)
    y = np.empty(n, np.float64)
    _check(_L().gg_points2d(n, seed, _ptr(x), _ptr(y)), "points2d")
    return x, y


def knn2d(n: int, k: int = 10, seed: int = 3):
    """Directed k-NN graph of n uniform points in the unit square (n*k pairs)."""
    src = np.empty(n * k, np.int32)
    dst = np.empty(n * k, np.int32)
    _check(_L().gg_knn2d(n, k, seed, _ptr(src), _ptr(dst)), "knn2d")
    return src, dst


def clique_sizes(n: int, count: int = 64, smin: int = 50, smax: int = 2000, seed: int = 4):
    sizes = np.empty(count, np.int32)
    _check(_L().gg_cliques(n, count, smin, smax, seed, _ptr(sizes), None, None, None), "cliques")
    return sizes


def planted_cliques(n: int, count: int = 64, smin: int = 50, smax: int = 2000, seed: int = 4):
    """Returns (src, dst, sizes, members): all pairs of each planted clique."""
    sizes = clique_sizes(n, count, smin, smax, seed)
    pairs = int(sum(int(s) * (int(s) - 1) // 2 for s in sizes))
    src = np.empty(pairs, np.int32)
    dst = np.empty(pairs, np.int32)
    members = np.empty(int(sizes.sum()), np.int32)
    _check(_L().gg_cliques(n, count, smin, smax, seed, _ptr(sizes), _ptr(members), _ptr(src),
                           _ptr(dst)), "cliques")
    return src, dst, sizes, members


def permutation(n: int, seed: int):
    p = np.empty(n, np.int32)
    _check(_L().gg_permutation(n, seed, _ptr(p)), "permutation")
    return p


# --------------------------------------------------------------------------- workloads
def workload_er10k():
    """ER G(n=10,000, m=50,000), seed 1."""
    n = 10_000
    s, d = er(n, 50_000, seed=1)
    return n, s, d


def workload_rmat(scale: int = 24, edge_factor: int = 16):
    """R-MAT scale 24, edge factor 16, (a,b,c,d) = (.57,.19,.19,.05), ids permuted
    (seed 1 for edges, seed 2 for the permutation)."""
    n = 1 << scale
    s, d = rmat(scale, edge_factor, seed=1, perm_seed=2)
    return n, s, d


def workload_knn_cliques(n: int = 1 << 24, k: int = 10, cliques: int = 64,
                         smin: int = 50, smax: int = 2000):
    """Undirected 10-NN graph of n points (seed 3) plus planted cliques (seed 4)."""
    s1, d1 = knn2d(n, k, seed=3)
    s2, d2, sizes, members = planted_cliques(n, cliques, smin, smax, seed=4)
    return n, np.concatenate([s1, s2]), np.concatenate([d1, d2]), sizes, members


def batch_spec(G: int = 4096, nmin: int = 1000, nmax: int = 200_000, dmin: float = 4.0,
               dmax: float = 64.0, seed: int = 5):
    """Per-graph (n, m, kind, seed) rows of the batched workload: n log-uniform,
    average degree uniform, ER or R-MAT with probability 1/2; graph g uses seed+g."""
    spec = np.empty((G, 4), np.int64)
    _check(_L().gg_batch_spec(G, nmin, nmax, dmin, dmax, seed, _ptr(spec)), "batch_spec")
    return spec


def batch_edges(spec: np.ndarray):
    """Edges of every graph in spec, concatenated (graph-local ids).
    Returns (eoff[G+1], src, dst)."""
    spec = np.ascontiguousarray(spec, dtype=np.int64)
    G = spec.shape[0]
    eoff = np.zeros(G + 1, np.int64)
    np.cumsum(spec[:, 1], out=eoff[1:])
    src = np.empty(int(eoff[-1]), np.int32)
    dst = np.empty(int(eoff[-1]), np.int32)
    a, b, c = RMAT_ABC
    _check(_L().gg_batch_edges(G, _ptr(spec), _ptr(eoff), a, b, c, _ptr(src), _ptr(dst)),
           "batch_edges")
    return eoff, src, dst


# --------------------------------------------------------------------------- closed forms
def _pairs(lst):
    if not lst:
        return np.empty(0, np.int32), np.empty(0, np.int32)
    a = np.asarray(lst, dtype=np.int64)
    return a[:, 0].astype(np.int32), a[:, 1].astype(np.int32)


def complete(n: int):
    i, j = np.triu_indices(n, 1)
    return n, i.astype(np.int32), j.astype(np.int32)


def path(n: int):
    i = np.arange(n - 1, dtype=np.int32)
    return n, i, i + 1


def star(leaves: int):
    return leaves + 1, np.zeros(leaves, np.int32), np.arange(1, leaves + 1, dtype=np.int32)


def cycle(n: int):
    i = np.arange(n, dtype=np.int32)
    return n, i, ((i + 1) % n).astype(np.int32)


def complete_bipartite(a: int, b: int):
    i, j = np.meshgrid(np.arange(a), np.arange(a, a + b), indexing="ij")
    return a + b, i.ravel().astype(np.int32), j.ravel().astype(np.int32)


def grid2d(a: int, b: int):
    idx = np.arange(a * b).reshape(a, b)
    s = np.concatenate([idx[:-1, :].ravel(), idx[:, :-1].ravel()])
    d = np.concatenate([idx[1:, :].ravel(), idx[:, 1:].ravel()])
    return a * b, s.astype(np.int32), d.astype(np.int32)


def grid3d(a: int, b: int, c: int):
    idx = np.arange(a * b * c).reshape(a, b, c)
    s = np.concatenate([idx[:-1].ravel(), idx[:, :-1].ravel(), idx[:, :, :-1].ravel()])
    d = np.concatenate([idx[1:].ravel(), idx[:, 1:].ravel(), idx[:, :, 1:].ravel()])
    return a * b * c, s.astype(np.int32), d.astype(np.int32)


def random_tree(n: int, seed: int):
    """Random recursive tree: vertex i > 0 attaches to a uniform earlier vertex."""
    rng = np.random.default_rng(seed)
    if n < 2:
        return n, np.empty(0, np.int32), np.empty(0, np.int32)
    parent = (rng.random(n - 1) * np.arange(1, n)).astype(np.int64)
    return n, np.arange(1, n, dtype=np.int32), parent.astype(np.int32)


def staircase(K: int):
    """Clique on K+1 vertices [0, K] plus vertices v_i = K+i (1 <= i < K) each
    joined to clique vertices 0..i-1: the HCNS shape of Sec. 6.1 with one
    vertex per coreness value 1..K-1 and a dense core of coreness K."""
    n, s, d = complete(K + 1)
    ss, dd = [s], [d]
    for i in range(1, K):
        ss.append(np.full(i, K + i, np.int32))
        dd.append(np.arange(i, dtype=np.int32))
    return 2 * K, np.concatenate(ss), np.concatenate(dd)


def disjoint_union(*graphs):
    """Concatenates (n, src, dst) graphs with relabelled ids."""
    base = 0
    ss, dd = [], []
    for n, s, d in graphs:
        ss.append(np.asarray(s, np.int64) + base)
        dd.append(np.asarray(d, np.int64) + base)
        base += n
    s = np.concatenate(ss) if ss else np.empty(0, np.int64)
    d = np.concatenate(dd) if dd else np.empty(0, np.int64)
    return base, s.astype(np.int32), d.astype(np.int32)


def small_random(n: int, m: int, seed: int, loops: bool = True):
    """Tiny multigraph edge list with duplicates, reversed pairs and (optionally)
    self-loops, for exercising CSR builders."""
    rng = np.random.default_rng(seed)
    s = rng.integers(0, max(n, 1), m).astype(np.int32)
    d = rng.integers(0, max(n, 1), m).astype(np.int32)
    if not loops:
        keep = s != d
        s, d = s[keep], d[keep]
    return n, s, d


