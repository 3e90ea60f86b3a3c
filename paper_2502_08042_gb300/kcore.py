"""Python binding of libkcore (include/kcore.h): argument marshalling only.

Device arrays are torch CUDA tensors (PyTorch supplies device memory and
streams); every step of the decomposition runs in the library's kernels. There
is no fallback: if the library cannot be built or loaded, or a call fails, an
exception is raised.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _native

STATUS = {0: "OK", 1: "INVALID", 2: "OOM", 3: "CUDA", 4: "TIMEOUT", 5: "NOT_SIMPLE", 6: "CAPACITY"}
OPTIONS = {"sync_mode": 0, "ctas_per_sm": 1, "slice_arcs": 2, "local_queue": 3, "timeout_ms": 4,
           "min_ctas": 5, "vertices_per_cta": 6, "test_stall": 7,
           "trace": 8, "idle_sleep_ns": 9, "poll_sleep_ns": 10, "batch_block": 11,
           "batch_smem_vertices": 12, "batch_ctas_per_sm": 13, "local_batches": 14, "level_window": 15,
           "batch_update": 16, "sampling": 17, "sample_mu": 18, "sample_threshold": 19, "sample_seed": 20,
           "sample_check": 21, "warp_combine": 22, "precheck_items": 23, "tail_items": 24,
           "tail_entries": 25, "park_sleep_ns": 26, "scan_entries": 27, "batch_cluster": 28,
           "batch_big_arcs": 29}
TRACE_FIELDS = ("t_start", "t_scanned", "t_done", "level", "scanned", "found", "queued", "scan_ctas",
                "arcs", "decrements", "max_cta_scan_ns", "max_cta_start_delay_ns", "busy_ns",
                "batches")


class KCoreError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"kcore {STATUS.get(status, status)}: {message}")
        self.status = status
        self.code = STATUS.get(status, str(status))


def _torch():
    import torch
    return torch


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        return t.ctypes.data if t.size else None
    return t.data_ptr() if t.numel() else None


def _stream_ptr(stream) -> int | None:
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream or None


class KCore:
    """One library handle bound to one CUDA device (not thread-safe)."""

    def __init__(self, device: int = 0, **options):
        self._L = _native.lib()
        self.device = device
        h = ctypes.c_void_p()
        st = self._L.kcore_create(ctypes.byref(h), device)
        if st != 0:
            raise KCoreError(st, f"kcore_create(device={device}) failed")
        self._h = h
        for k, v in options.items():
            self.set_option(k, v)

    # ------------------------------------------------------------ plumbing
    def _check(self, st: int):
        if st != 0:
            msg = self._L.kcore_last_error(self._h)
            raise KCoreError(st, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "_h", None):
            self._L.kcore_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def set_option(self, name: str, value: int):
        self._check(self._L.kcore_set_option(self._h, OPTIONS[name], int(value)))

    def get_option(self, name: str) -> int:
        v = ctypes.c_int64()
        self._check(self._L.kcore_get_option(self._h, OPTIONS[name], ctypes.byref(v)))
        return int(v.value)

    def workspace_size(self, n: int, m: int) -> int:
        b = ctypes.c_size_t()
        self._check(self._L.kcore_workspace_size(self._h, n, m, ctypes.byref(b)))
        return int(b.value)

    def set_workspace(self, buf) -> None:
        """Uses a caller-owned device buffer (e.g. a torch uint8 tensor) as
        workspace; None returns to library-owned memory."""
        if buf is None:
            self._check(self._L.kcore_set_workspace(self._h, None, 0))
        else:
            self._check(self._L.kcore_set_workspace(self._h, buf.data_ptr(), buf.numel() * buf.element_size()))
        self._ws_ref = buf

    def sync(self) -> None:
        """Waits for the last call and raises if the device reported an error."""
        self._check(self._L.kcore_sync_status(self._h))

    def stats(self) -> dict:
        s = _native.Stats()
        self._check(self._L.kcore_get_stats(self._h, ctypes.byref(s)))
        return {f: int(getattr(s, f)) for f, _ in _native.Stats._fields_}

    def barrier_latency_ns(self, grid: int = 0, iters: int = 2000) -> float:
        """Mean time of one grid barrier of the bulk-synchronous schedule
        (grid CTAs, 0 = the large-graph grid), measured on the device."""
        v = ctypes.c_double()
        self._check(self._L.kcore_barrier_latency(self._h, int(grid), int(iters), ctypes.byref(v)))
        return float(v.value)

    def trace(self) -> np.ndarray:
        """Timeline of the last decomposition: one row of TRACE_FIELDS per
        round with trace=1, one row per phase with trace=2 (fields as
        kcore_get_trace documents)."""
        st = self.stats()
        max_r = max(st["barriers"] + st["tail_phases"] if self.get_option("trace") == 2 else st["rounds"], 0)
        buf = np.zeros((max(max_r, 1), len(TRACE_FIELDS)), np.uint64)
        got = ctypes.c_int64()
        self._check(self._L.kcore_get_trace(self._h, buf.ctypes.data, max_r, ctypes.byref(got)))
        return buf[:got.value]

    # ------------------------------------------------------------ compute
    def decompose(self, offsets, adj, coreness=None, kmax=None, stream=None, sync: bool = True):
        """Coreness of every vertex of a simple undirected CSR held on the GPU.

        offsets: int64 CUDA tensor [n+1]; adj: int32 CUDA tensor [m].
        Returns (coreness int32 [n], kmax int32 [1]) CUDA tensors. With
        sync=False the call only queues work (check errors with sync())."""
        torch = _torch()
        n = offsets.numel() - 1
        m = adj.numel()
        assert offsets.dtype == torch.int64 and adj.dtype == torch.int32
        assert offsets.is_cuda and adj.is_cuda and offsets.is_contiguous() and adj.is_contiguous()
        if coreness is None:
            coreness = torch.empty(max(n, 0), dtype=torch.int32, device=offsets.device)
        if kmax is None:
            kmax = torch.empty(1, dtype=torch.int32, device=offsets.device)
        st = self._L.kcore_decompose(self._h, n, m, _ptr(offsets), _ptr(adj), _ptr(coreness),
                                     _ptr(kmax), _stream_ptr(stream))
        self._check(st)
        if sync:
            self.sync()
        return coreness, kmax

    def core_mask(self, offsets, adj, kprime: int, mask=None, size=None, stream=None, sync: bool = True):
        """Membership of every vertex in the k'-core (int32 1/0 CUDA tensor
        [n]) and the k'-core's vertex count (int64 CUDA tensor [1])."""
        torch = _torch()
        n = offsets.numel() - 1
        m = adj.numel()
        assert offsets.dtype == torch.int64 and adj.dtype == torch.int32
        assert offsets.is_cuda and adj.is_cuda and offsets.is_contiguous() and adj.is_contiguous()
        if mask is None:
            mask = torch.empty(max(n, 0), dtype=torch.int32, device=offsets.device)
        if size is None:
            size = torch.empty(1, dtype=torch.int64, device=offsets.device)
        self._check(self._L.kcore_core_mask(self._h, n, m, _ptr(offsets), _ptr(adj), int(kprime), _ptr(mask),
                                            _ptr(size), _stream_ptr(stream)))
        if sync:
            self.sync()
        return mask, size

    def validate_csr(self, offsets, adj, stream=None, sync: bool = True) -> None:
        """Checks on the GPU that (offsets, adj) is a simple undirected CSR
        (offsets sound, ids in range, no self-loops, ascending lists,
        symmetric). With sync, raises KCoreError (code NOT_SIMPLE) naming the
        first failure; stats() then holds invalid_check/_vertex/_arc."""
        torch = _torch()
        n = offsets.numel() - 1
        m = adj.numel()
        assert offsets.dtype == torch.int64 and adj.dtype == torch.int32
        assert offsets.is_cuda and adj.is_cuda and offsets.is_contiguous() and adj.is_contiguous()
        self._check(self._L.kcore_validate_csr(self._h, n, m, _ptr(offsets), _ptr(adj), _stream_ptr(stream)))
        if sync:
            self.sync()

    def decompose_batched(self, graph_vertex_offsets, offsets, adj, coreness=None, kmax=None,
                          stream=None, sync: bool = True):
        """Coreness of every graph of a segmented CSR on the GPU (graph-local
        adjacency ids). graph_vertex_offsets: int64 [G+1]; offsets: int64 [N+1];
        adj: int32 [M]. Returns (coreness int32 [N], kmax int32 [G])."""
        torch = _torch()
        G = graph_vertex_offsets.numel() - 1
        N = offsets.numel() - 1
        M = adj.numel()
        dev = offsets.device
        if coreness is None:
            coreness = torch.empty(max(N, 0), dtype=torch.int32, device=dev)
        if kmax is None:
            kmax = torch.empty(max(G, 0), dtype=torch.int32, device=dev)
        self._check(self._L.kcore_decompose_batched(
            self._h, G, N, M, _ptr(graph_vertex_offsets), _ptr(offsets), _ptr(adj), _ptr(coreness),
            _ptr(kmax), _stream_ptr(stream)))
        if sync:
            self.sync()
        return coreness, kmax

    def autotune(self, offsets, adj, coreness=None, kmax=None, repeats: int = 2, stream=None):
        """Times the single-graph peel's candidate schedules on this graph,
        keeps the fastest in the handle's options and returns (coreness, kmax,
        tuning dict) computed with it."""
        torch = _torch()
        n = offsets.numel() - 1
        dev = offsets.device
        if coreness is None:
            coreness = torch.empty(max(n, 0), dtype=torch.int32, device=dev)
        if kmax is None:
            kmax = torch.empty(1, dtype=torch.int32, device=dev)
        t = _native.Tuning()
        self._check(self._L.kcore_autotune(self._h, n, adj.numel(), _ptr(offsets), _ptr(adj), _ptr(coreness),
                                           _ptr(kmax), int(repeats), ctypes.byref(t), _stream_ptr(stream)))
        return coreness, kmax, {f: getattr(t, f) for f, _ in t._fields_}

    def autotune_batched(self, graph_vertex_offsets, offsets, adj, coreness=None, kmax=None,
                         repeats: int = 2, stream=None):
        """Times the batched peel's launch shapes on this batch, keeps the
        fastest in the handle's options and returns (coreness, kmax, tuning
        dict) computed with it."""
        torch = _torch()
        G = graph_vertex_offsets.numel() - 1
        N = offsets.numel() - 1
        M = adj.numel()
        dev = offsets.device
        if coreness is None:
            coreness = torch.empty(max(N, 0), dtype=torch.int32, device=dev)
        if kmax is None:
            kmax = torch.empty(max(G, 0), dtype=torch.int32, device=dev)
        t = _native.BatchTuning()
        self._check(self._L.kcore_autotune_batched(
            self._h, G, N, M, _ptr(graph_vertex_offsets), _ptr(offsets), _ptr(adj), _ptr(coreness),
            _ptr(kmax), int(repeats), ctypes.byref(t), _stream_ptr(stream)))
        return coreness, kmax, {f: getattr(t, f) for f, _ in t._fields_}

    def build_csr_batched(self, graph_vertex_offsets, graph_edge_offsets, src, dst,
                          max_graph_vertices: int, stream=None, sync: bool = True):
        """Segmented CSR of a batch of edge lists with graph-local ids (all CUDA
        tensors; offsets int64). Returns (offsets int64 [N+1], adj int32 [m])."""
        torch = _torch()
        G = graph_vertex_offsets.numel() - 1
        N = int(graph_vertex_offsets[-1].item())
        E = src.numel()
        dev = src.device
        off = torch.empty(N + 1, dtype=torch.int64, device=dev)
        adj = torch.empty(max(2 * E, 1), dtype=torch.int32, device=dev)
        m = torch.zeros(1, dtype=torch.int64, device=dev)
        self._check(self._L.kcore_build_csr_batched(
            self._h, G, N, E, int(max_graph_vertices), _ptr(graph_vertex_offsets),
            _ptr(graph_edge_offsets), _ptr(src), _ptr(dst), _ptr(off), _ptr(adj), _ptr(m),
            _stream_ptr(stream)))
        if not sync:
            return off, adj, m
        self.sync()
        return off, adj[: int(m.item())]

    def batched_workspace_size(self, G: int, N: int) -> int:
        b = ctypes.c_size_t()
        self._check(self._L.kcore_batched_workspace_size(self._h, G, N, ctypes.byref(b)))
        return int(b.value)

    def build_csr(self, n: int, src, dst, stream=None, sync: bool = True):
        """Simple undirected CSR of a device edge list (int32 tensors).
        Returns (offsets int64 [n+1], adj int32 [m]) CUDA tensors; with
        sync=False returns (offsets, adj_buffer [2E], m_tensor) without waiting."""
        torch = _torch()
        E = src.numel()
        assert dst.numel() == E and src.dtype == torch.int32 and dst.dtype == torch.int32
        dev = src.device
        off = torch.empty(n + 1, dtype=torch.int64, device=dev)
        adj = torch.empty(max(2 * E, 1), dtype=torch.int32, device=dev)
        m = torch.zeros(1, dtype=torch.int64, device=dev)
        self._check(self._L.kcore_build_csr(self._h, n, E, _ptr(src), _ptr(dst), _ptr(off), _ptr(adj),
                                            _ptr(m), _stream_ptr(stream)))
        if not sync:
            return off, adj, m
        self.sync()
        return off, adj[: int(m.item())]

    def build_csr_workspace_size(self, n: int, E: int) -> int:
        b = ctypes.c_size_t()
        self._check(self._L.kcore_build_csr_workspace_size(self._h, n, E, ctypes.byref(b)))
        return int(b.value)

    def decompose_host(self, offsets: np.ndarray, adj: np.ndarray, stream=None):
        """End-to-end call on host arrays: H2D copies, peel, D2H copies, wait.
        Returns (coreness int32 numpy [n], kmax int)."""
        offsets = np.ascontiguousarray(offsets, dtype=np.int64)
        adj = np.ascontiguousarray(adj, dtype=np.int32)
        n = len(offsets) - 1
        core = np.empty(n, np.int32)
        km = np.zeros(1, np.int32)
        st = self._L.kcore_decompose_host(self._h, n, len(adj), _ptr(offsets), _ptr(adj),
                                          _ptr(core), _ptr(km), _stream_ptr(stream))
        self._check(st)
        return core, int(km[0])

    def decompose_host_into(self, offsets, adj, core_out, kmax_out, stream=None):
        """decompose_host with caller-provided (e.g. pinned) host buffers."""
        st = self._L.kcore_decompose_host(self._h, len(offsets) - 1, len(adj), _ptr(offsets),
                                          _ptr(adj), _ptr(core_out), _ptr(kmax_out),
                                          _stream_ptr(stream))
        self._check(st)


class KCoreServer:
    """Request loop with continuous batching (kcore_server_*). Host arrays given
    to submit() must stay alive until their ticket comes back from poll().
    The arguments mirror kcore_server_config (0 = its default): batch_cluster
    is the cluster size for the largest graphs of a batched launch (2, 4 or 8;
    1 = one CTA per graph; default 4), batch_big_arcs the arcs from which a
    graph takes a cluster (default: the launch's arcs per CTA)."""

    def __init__(self, device: int = 0, pool_bytes: int = 0, max_requests: int = 0, streams: int = 0,
                 large_vertices: int = 0, large_arcs: int = 0, batch_cluster: int = 0, batch_big_arcs: int = 0):
        self._L = _native.lib()
        cfg = _native.ServerConfig(pool_bytes, max_requests, streams, large_vertices, large_arcs, batch_cluster,
                                   batch_big_arcs)
        h = ctypes.c_void_p()
        st = self._L.kcore_server_create(ctypes.byref(h), device, ctypes.byref(cfg))
        if st != 0:
            raise KCoreError(st, "kcore_server_create failed")
        self._h = h
        self._keep = {}
        self._cap = max_requests or 4096
        self._t = np.zeros(self._cap, np.int64)
        self._k = np.zeros(self._cap, np.int32)
        self._s = np.zeros(self._cap, np.int32)

    def submit(self, offsets: np.ndarray, adj: np.ndarray, coreness_out: np.ndarray):
        """Queues a host CSR; returns its ticket, or None when not admitted now."""
        n = len(offsets) - 1
        t = ctypes.c_int64()
        st = self._L.kcore_server_submit(self._h, n, len(adj), _ptr(offsets), _ptr(adj),
                                         _ptr(coreness_out), ctypes.byref(t))
        if st == 6:  # KCORE_ERR_CAPACITY: pool or slots full
            return None
        if st != 0:
            raise KCoreError(st, "kcore_server_submit failed")
        self._keep[t.value] = (offsets, adj, coreness_out)
        return t.value

    def poll(self):
        """Advances all requests; returns a list of (ticket, kmax, status)."""
        cnt = ctypes.c_int()
        st = self._L.kcore_server_poll(self._h, self._t.ctypes.data, self._k.ctypes.data,
                                       self._s.ctypes.data, self._cap, ctypes.byref(cnt))
        if st != 0:
            raise KCoreError(st, "kcore_server_poll failed")
        out = []
        for i in range(cnt.value):
            t = int(self._t[i])
            self._keep.pop(t, None)
            out.append((t, int(self._k[i]), int(self._s[i])))
        return out

    def info(self):
        a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        self._L.kcore_server_info(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c))
        return {"in_flight": a.value, "pool_used": b.value, "pool_bytes": c.value}

    def close(self):
        if getattr(self, "_h", None):
            self._L.kcore_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def decompose(offsets, adj, device: int | None = None, **options):
    """One-shot convenience wrapper around KCore.decompose (synchronous)."""
    dev = offsets.device.index if device is None else device
    with KCore(dev or 0, **options) as k:
        return k.decompose(offsets, adj)
