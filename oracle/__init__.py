"""CPU oracle for exact k-core decomposition (arXiv 2502.08042).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, by ``__graft_entry__.smoke()``
and by the CPU-baseline leg of ``bench.py``. The library never imports it, and
it shares no code with the CUDA path.

Coreness (Sec. 2, "Notations"): the k-core is the largest subgraph with minimum
degree >= k; the coreness of v is the largest k with v in the k-core. The C
routines (``kcore_oracle.c``) compute it by Batagelj-Zaversnik, by
Algorithm 1 with the sequential Peel and by Algorithm 4 with the sampling Peel
of Algorithm 5 (Philox coins), and check any claimed answer with a
certificate; ``brute.py`` recomputes it from the definition for tiny graphs.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

from .brute import brute_coreness  # noqa: F401  (re-export)

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libkcore_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compiles kcore_oracle.c with the host gcc into _build/libkcore_oracle.so."""
    src = os.path.join(_HERE, "kcore_oracle.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, src])
    os.replace(tmp, _SO)
    return _SO


def _L():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64, p = ctypes.c_int64, ctypes.c_void_p
            lib.oc_build_csr.argtypes = [i64, i64, p, p, p, p]
            lib.oc_build_csr.restype = i64
            lib.oc_check_simple.argtypes = [i64, p, p]
            lib.oc_check_simple.restype = ctypes.c_int
            lib.oc_bz.argtypes = [i64, p, p, p]
            lib.oc_bz.restype = ctypes.c_int
            lib.oc_alg1.argtypes = [i64, p, p, p, p]
            lib.oc_alg1.restype = ctypes.c_int
            lib.oc_check.argtypes = [i64, p, p, p, p]
            lib.oc_check.restype = ctypes.c_int
            lib.oc_kcore_mask.argtypes = [i64, p, p, ctypes.c_int32, p]
            lib.oc_kcore_mask.restype = i64
            lib.oc_philox4x32_10.argtypes = [p, p, p]
            lib.oc_philox4x32_10.restype = None
            lib.oc_kcore_sampled.argtypes = [i64, p, p, i64, i64, ctypes.c_uint64, p, p]
            lib.oc_kcore_sampled.restype = ctypes.c_int
            _lib = lib
    return _lib


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def build_csr(n: int, src, dst):
    """Simple undirected CSR (int64 offsets[n+1], int32 adj) of an edge list:
    both directions, self-loops dropped, duplicates kept once, lists ascending."""
    src = _c(src, np.int32)
    dst = _c(dst, np.int32)
    off = np.zeros(n + 1, np.int64)
    adj = np.empty(max(2 * len(src), 1), np.int32)
    m = _L().oc_build_csr(n, len(src), src.ctypes.data, dst.ctypes.data, off.ctypes.data,
                          adj.ctypes.data)
    if m < 0:
        raise ValueError(f"oracle.build_csr failed ({m})")
    return off, adj[:m].copy()


def check_simple(n: int, off, adj) -> int:
    """0 when (off, adj) is a simple undirected CSR, else a positive code."""
    off = _c(off, np.int64)
    adj = _c(adj, np.int32)
    return int(_L().oc_check_simple(n, off.ctypes.data, adj.ctypes.data if len(adj) else None))


def bz(n: int, off, adj):
    """Coreness by the Batagelj-Zaversnik bucket peel (int32[n])."""
    off = _c(off, np.int64)
    adj = _c(adj, np.int32)
    core = np.zeros(n, np.int32)
    rc = _L().oc_bz(n, off.ctypes.data, adj.ctypes.data if len(adj) else None, core.ctypes.data)
    if rc:
        raise MemoryError("oracle.bz")
    return core


ALG1_STATS = ("rounds", "subrounds", "sum_active", "frontier_inserts", "kmax", "nonempty_rounds")


def alg1(n: int, off, adj):
    """Coreness by Algorithm 1 with the sequential Peel; returns (core, stats)."""
    off = _c(off, np.int64)
    adj = _c(adj, np.int32)
    core = np.full(n, -1, np.int32)
    st = np.zeros(6, np.int64)
    rc = _L().oc_alg1(n, off.ctypes.data, adj.ctypes.data if len(adj) else None, core.ctypes.data,
                      st.ctypes.data)
    if rc:
        raise MemoryError("oracle.alg1")
    return core, dict(zip(ALG1_STATS, (int(x) for x in st)))


def check(n: int, off, adj, core):
    """Certificate check of a claimed coreness vector: (code, bad_vertex);
    code 0 means the vector is the coreness."""
    off = _c(off, np.int64)
    adj = _c(adj, np.int32)
    core = _c(core, np.int32)
    bad = ctypes.c_int64(-1)
    rc = _L().oc_check(n, off.ctypes.data, adj.ctypes.data if len(adj) else None,
                       core.ctypes.data, ctypes.byref(bad))
    if rc < 0:
        raise MemoryError("oracle.check")
    return int(rc), int(bad.value)


def kcore_mask(n: int, off, adj, kprime: int):
    """Membership of every vertex in the k'-core (App. B): int32 1/0 by
    repeated deletion of vertices whose remaining degree is below kprime.
    Returns (mask, size)."""
    off = _c(off, np.int64)
    adj = _c(adj, np.int32)
    mask = np.zeros(max(n, 0), np.int32)
    size = _L().oc_kcore_mask(n, off.ctypes.data, adj.ctypes.data if len(adj) else None, int(kprime),
                              mask.ctypes.data)
    if size < 0:
        raise MemoryError("oracle.kcore_mask")
    return mask, int(size)


def philox4x32_10(ctr, key):
    """Philox4x32-10 (Salmon et al., SC 2011) of a 4-word counter and a 2-word
    key: the four output words."""
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (ctypes.c_uint32 * 4)()
    _L().oc_philox4x32_10(c, k, o)
    return tuple(int(x) for x in o)


SAMPLED_STATS = ("sampled_at_start", "recounts", "bag_inserts", "failed_validations", "heads",
                 "miss_round", "miss_vertex", "rounds")


def kcore_sampled(n: int, off, adj, mu: int, threshold: int, seed: int = 0):
    """Algorithm 4 with the sampling Peel of Algorithm 5 (Sec. 4.1), round by
    round. Returns (ok, core, stats): ok False when the recovery check found a
    vertex that missed an earlier round (core is then incomplete)."""
    off = _c(off, np.int64)
    adj = _c(adj, np.int32)
    core = np.full(max(n, 0), -1, np.int32)
    st = np.zeros(8, np.int64)
    rc = _L().oc_kcore_sampled(n, off.ctypes.data, adj.ctypes.data if len(adj) else None, int(mu),
                               int(threshold), ctypes.c_uint64(int(seed) & (2**64 - 1)), core.ctypes.data,
                               st.ctypes.data)
    if rc < 0:
        raise MemoryError("oracle.kcore_sampled")
    return rc == 0, core, dict(zip(SAMPLED_STATS, (int(x) for x in st)))


def kmax(core) -> int:
    return int(core.max()) if len(core) else 0


def bz_batch(gv, off, adj, threads: int | None = None, graphs=None):
    """Per-graph BZ over a segmented CSR (graph g owns vertices [gv[g], gv[g+1]),
    arcs with graph-local ids). Runs graphs in parallel on host threads.
    Returns (core[N], kmax[G]) for all graphs, or for the listed ``graphs``
    (other entries left at -1)."""
    gv = _c(gv, np.int64)
    off = _c(off, np.int64)
    adj = _c(adj, np.int32)
    G = len(gv) - 1
    core = np.full(int(gv[-1]), -1, np.int32)
    km = np.full(G, -1, np.int32)
    todo = range(G) if graphs is None else graphs

    def one(g):
        a, b = int(gv[g]), int(gv[g + 1])
        o = off[a:b + 1] - off[a]
        ad = adj[off[a]:off[b]]
        c = bz(b - a, o, ad)
        core[a:b] = c
        km[g] = kmax(c)

    with ThreadPoolExecutor(max_workers=threads or os.cpu_count() or 1) as ex:
        list(ex.map(one, todo))
    return core, km
