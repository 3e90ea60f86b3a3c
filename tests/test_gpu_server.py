"""The served peel (kcore_server_*): every request's coreness and k_max are the
oracle's, and the same whether the request runs alone or mixed with others
that arrive while it is on the GPU; admission by pool size defers requests
without losing any."""
import time

import numpy as np
import pytest

import graphgen as gg
import oracle
from tests.batch_util import spec_batch

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2502_08042_gb300 import KCoreServer  # noqa: E402


def make_requests():
    spec, eoff, s, d, ns, lists = spec_batch(24, nmin=500, nmax=40000, seed=8)
    reqs = []
    for n, (ss, dd) in zip(ns, lists):
        off, adj = oracle.build_csr(int(n), ss, dd)
        reqs.append((off, adj))
    # a larger R-MAT graph and closed forms
    rs, rd = gg.rmat(17, 16, seed=3, perm_seed=4)
    reqs.append(oracle.build_csr(1 << 17, rs, rd))
    for n, a, b in (gg.staircase(70), gg.complete(40), gg.path(5000)):
        reqs.append(oracle.build_csr(n, a, b))
    reqs.append((np.zeros(1, np.int64), np.zeros(0, np.int32)))  # empty graph
    return reqs


def run_all(server, reqs, order, burst):
    """Submits in `order`, `burst` at a time, polling in between; returns
    {index: (core, kmax, status)}."""
    outs = {i: np.full(max(len(reqs[i][0]) - 1, 1), -9, np.int32) for i in range(len(reqs))}
    ticket_of, res = {}, {}
    pending = list(order)
    deadline = time.time() + 120
    while (pending or ticket_of) and time.time() < deadline:
        for _ in range(burst):
            if not pending:
                break
            i = pending[0]
            off, adj = reqs[i]
            t = server.submit(off, adj, outs[i])
            if t is None:
                break  # not admitted now: retry after completions
            ticket_of[t] = i
            pending.pop(0)
        for t, km, st in server.poll():
            i = ticket_of.pop(t)
            res[i] = (outs[i][: len(reqs[i][0]) - 1].copy(), km, st)
    assert not pending and not ticket_of, "requests left unfinished"
    return res


def test_server_alone_and_mixed_match_oracle():
    reqs = make_requests()
    want = [oracle.bz(len(o) - 1, o, a) for o, a in reqs]
    # force the whole-GPU path for the R-MAT request (> 100k vertices)
    with KCoreServer(0, pool_bytes=1 << 30, large_vertices=100_000) as srv:
        alone = {}
        for i in range(len(reqs)):
            alone.update(run_all(srv, reqs, [i], 1))
        rng = np.random.default_rng(1)
        order = list(rng.permutation(len(reqs)))
        mixed = run_all(srv, reqs, order, 5)
    for i, w in enumerate(want):
        for res in (alone, mixed):
            core, km, st = res[i]
            assert st == 0
            np.testing.assert_array_equal(core, w)
            assert km == (int(w.max()) if len(w) else 0)
        np.testing.assert_array_equal(alone[i][0], mixed[i][0])


def test_server_admission_defers_without_loss():
    reqs = make_requests()[:20]
    want = [oracle.bz(len(o) - 1, o, a) for o, a in reqs]
    biggest = max(8 * len(o) + 4 * len(a) + 24 * len(o) for o, a in reqs)
    # a pool for about two requests at a time: most submissions are deferred
    with KCoreServer(0, pool_bytes=2 * biggest + (1 << 20), max_requests=8) as srv:
        res = run_all(srv, reqs, list(range(len(reqs))), len(reqs))
        assert srv.info()["in_flight"] == 0
    for i, w in enumerate(want):
        np.testing.assert_array_equal(res[i][0], w)


@pytest.mark.parametrize("cluster", [1, 2, 8])
def test_server_cluster_settings_match_oracle(cluster):
    """Batched launches with one CTA per graph (1) or clusters of 2 or 8 CTAs
    for their largest graphs (listed first): the same exact results, with the
    R-MAT request kept on the batched path (large_vertices above it) and the
    threshold forcing clusters onto every graph with arcs (big arcs 1)."""
    reqs = make_requests()
    want = [oracle.bz(len(o) - 1, o, a) for o, a in reqs]
    for big in (0, 1):
        with KCoreServer(0, pool_bytes=1 << 30, large_vertices=1 << 20, batch_cluster=cluster,
                         batch_big_arcs=big) as srv:
            rng = np.random.default_rng(cluster + big)
            res = run_all(srv, reqs, list(rng.permutation(len(reqs))), 8)
        for i, w in enumerate(want):
            core, km, st = res[i]
            assert st == 0
            np.testing.assert_array_equal(core, w)
            assert km == (int(w.max()) if len(w) else 0)


def test_server_rejects_bad_cluster_settings():
    from paper_2502_08042_gb300 import KCoreError
    for bad in (3, 16, -2):
        with pytest.raises(KCoreError):
            KCoreServer(0, pool_bytes=1 << 26, batch_cluster=bad)
    with pytest.raises(KCoreError):
        KCoreServer(0, pool_bytes=1 << 26, batch_big_arcs=-1)
