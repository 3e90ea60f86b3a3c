"""Coreness straight from its definition, for tiny graphs (pure Python).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

For each k = 0, 1, 2, ... the k-core is obtained by repeatedly deleting every
vertex whose degree among the remaining vertices is below k until none is
left to delete (what remains is the largest subgraph of minimum degree >= k,
Sec. 2 "Notations"). The coreness of v is the largest k whose k-core still
contains v. Cost O(k_max * n * m): graphs of a few hundred edges at most.
"""
from __future__ import annotations


def k_core_members(n: int, nbrs: list[set[int]], k: int) -> set[int]:
    alive = set(range(n))
    changed = True
    while changed:
        changed = False
        for v in list(alive):
            if sum(1 for u in nbrs[v] if u in alive) < k:
                alive.discard(v)
                changed = True
    return alive


def brute_coreness(n: int, src, dst) -> list[int]:
    """Coreness of every vertex of the simple undirected graph spanned by the
    pairs (src[i], dst[i]) (self-loops ignored, repeated pairs counted once)."""
    nbrs: list[set[int]] = [set() for _ in range(n)]
    for a, b in zip(list(src), list(dst)):
        a, b = int(a), int(b)
        if a != b:
            nbrs[a].add(b)
            nbrs[b].add(a)
    core = [0] * n
    k = 1
    while True:
        members = k_core_members(n, nbrs, k)
        if not members:
            break
        for v in members:
            core[v] = k
        k += 1
    return core
