"""Segmented-CSR helpers for the batched tests (host side, oracle CSRs)."""
import numpy as np

import graphgen as gg
import oracle


def oracle_segmented(ns, edge_lists):
    """Segmented CSR from per-graph edge lists (local ids) with the oracle's
    CSR builder: (gv[G+1], off[N+1] global, adj local)."""
    G = len(ns)
    gv = np.zeros(G + 1, np.int64)
    np.cumsum(np.asarray(ns, np.int64), out=gv[1:])
    offs, adjs = [], []
    base = 0
    for n, (s, d) in zip(ns, edge_lists):
        o, a = oracle.build_csr(int(n), s, d)
        offs.append(o[:-1] + base)
        adjs.append(a)
        base += len(a)
    off = np.concatenate(offs + [np.array([base], np.int64)]) if G else np.zeros(1, np.int64)
    adj = np.concatenate(adjs) if adjs else np.zeros(0, np.int32)
    return gv, off.astype(np.int64), adj.astype(np.int32)


def spec_batch(G, nmin=1000, nmax=200_000, seed=5):
    """A batch with the batched workload's distribution (possibly smaller)."""
    spec = gg.batch_spec(G, nmin=nmin, nmax=nmax, seed=seed)
    eoff, s, d = gg.batch_edges(spec)
    ns = spec[:, 0].tolist()
    lists = [(s[eoff[g]:eoff[g + 1]], d[eoff[g]:eoff[g + 1]]) for g in range(G)]
    return spec, eoff, s, d, ns, lists
