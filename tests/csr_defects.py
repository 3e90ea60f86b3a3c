"""Plants one defect in a simple CSR (numpy, host side) for the tests of the
simple-CSR checks. Each insertion keeps every other list valid, so the defect
is the only failure and its check code, vertex and arc are known in advance.

Device check codes (kcore_validate_csr): 1 offsets not monotone or outside
[0, m], 2 offsets[0] != 0 or offsets[n] != m, 3 id outside [0, n), 4 self-loop,
5 list not strictly ascending, 6 arc without its reverse.
"""
import numpy as np

# device code -> the oracle's check_simple code for the same first failure
ORACLE_CODE = {1: 3, 2: 2, 3: 4, 4: 5, 5: 6, 6: 7}

KINDS = ("range_high", "range_negative", "self_loop", "repeat", "asymmetric")


def _insert(off, adj, v, pos, val):
    """adj with val inserted at index pos (inside or at the end of v's list)."""
    adj2 = np.insert(np.asarray(adj, np.int32), pos, np.int32(val))
    off2 = np.asarray(off, np.int64).copy()
    off2[v + 1:] += 1
    return off2, adj2


def plant(n, off, adj, kind, rng):
    """Returns (off2, adj2, code, vertex, arc) with exactly one defect of `kind`."""
    off = np.asarray(off, np.int64)
    adj = np.asarray(adj, np.int32)
    deg = np.diff(off)
    nz = np.flatnonzero(deg > 0)
    if kind == "range_high":  # id n appended at the end of v's list
        v = int(rng.choice(nz))
        pos = int(off[v + 1])
        o, a = _insert(off, adj, v, pos, n)
        return o, a, 3, v, pos
    if kind == "range_negative":  # -1 at the head of v's list (still ascending)
        v = int(rng.choice(nz))
        pos = int(off[v])
        o, a = _insert(off, adj, v, pos, -1)
        return o, a, 3, v, pos
    if kind == "self_loop":  # v in its own list, at its sorted place
        v = int(rng.integers(n))
        lst = adj[off[v]:off[v + 1]]
        pos = int(off[v] + np.searchsorted(lst, v))
        o, a = _insert(off, adj, v, pos, v)
        return o, a, 4, v, pos
    if kind == "repeat":  # an existing arc v->u stored twice
        v = int(rng.choice(nz))
        j = int(rng.integers(off[v], off[v + 1]))
        o, a = _insert(off, adj, v, j + 1, adj[j])
        return o, a, 5, v, j + 1
    if kind == "asymmetric":  # v->w with w not adjacent to v, reverse absent
        while True:
            v = int(rng.integers(n))
            w = int(rng.integers(n))
            lst = adj[off[v]:off[v + 1]]
            if w != v and not np.any(lst == w):
                break
        pos = int(off[v] + np.searchsorted(lst, w))
        o, a = _insert(off, adj, v, pos, w)
        return o, a, 6, v, pos
    raise ValueError(kind)
