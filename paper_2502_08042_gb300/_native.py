"""Builds and loads libkcore.so (the sm_103a CUDA library behind include/kcore.h).

The library is compiled in-tree with nvcc (one process per translation unit,
in parallel, then one link step) into ``_build/libkcore.so``. Loading never
falls back to anything else: a missing or unloadable library is an error.
"""
from __future__ import annotations

import ctypes
import glob
import os
import shutil
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
SO = os.path.join(BUILD, "libkcore.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

_lock = threading.Lock()
_lib = None


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libkcore")


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return _sources() + sorted(glob.glob(os.path.join(CSRC, "*.h"))) + \
        sorted(glob.glob(os.path.join(CSRC, "*.cuh"))) + sorted(glob.glob(os.path.join(INCLUDE, "*.h")))


def up_to_date() -> bool:
    if not os.path.exists(SO):
        return False
    t = os.path.getmtime(SO)
    return all(os.path.getmtime(p) <= t for p in _deps())


def build(force: bool = False, verbose: bool = False) -> str:
    """Compiles every csrc/*.cu for sm_103a and links _build/libkcore.so."""
    if not force and up_to_date():
        return SO
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE,
                    "-I", CSRC, "--expt-relaxed-constexpr"]
    if os.environ.get("KCORE_PTXAS_VERBOSE"):
        flags += ["-Xptxas", "-v"]

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src)[:-3] + ".o")
        r = subprocess.run([nvcc, *flags, "-c", src, "-o", obj], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and (r.stdout or r.stderr):
            print(r.stdout + r.stderr)
        return obj

    srcs = _sources()
    with ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 1))) as ex:
        objs = list(ex.map(compile_one, srcs))
    tmp = SO + f".tmp{os.getpid()}"
    r = subprocess.run([nvcc, *ARCH, "-shared", "-o", tmp, *objs], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, SO)
    return SO


def lib() -> ctypes.CDLL:
    """Loads libkcore.so (building it first when sources are newer)."""
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            _declare(L)
            _lib = L
    return _lib


c_i64, c_i32, c_p, c_sz = ctypes.c_int64, ctypes.c_int32, ctypes.c_void_p, ctypes.c_size_t


class Stats(ctypes.Structure):
    _fields_ = [(name, c_i64) for name in ("rounds", "empty_rounds", "items", "local_items",
                                           "scanned", "kmax", "grid", "sync_mode", "passes",
                                           "barriers", "batch_block", "batch_smem_vertices", "slice_arcs",
                                           "sample_vertices", "sample_recounts", "sample_bag",
                                           "sample_failed_validations", "sample_heads", "sample_reruns",
                                           "sample_miss_round", "invalid_check", "invalid_vertex", "invalid_arc",
                                           "tail_phases", "tail_episodes", "batch_cluster")]


class Tuning(ctypes.Structure):
    _fields_ = [("sync_mode", ctypes.c_int32), ("batch_update", ctypes.c_int32),
                ("warp_combine", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("tail_items", c_i64), ("tail_entries", c_i64), ("precheck_items", c_i64),
                ("local_batches", c_i64), ("candidates", ctypes.c_int32), ("ms", ctypes.c_double),
                ("cluster", ctypes.c_int32)]


class BatchTuning(ctypes.Structure):
    _fields_ = [("block", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("smem_vertices", ctypes.c_int32), ("candidates", ctypes.c_int32),
                ("ms", ctypes.c_double), ("cluster", ctypes.c_int32)]


# Every exported symbol of include/kcore.h with its ctypes signature.
SIGNATURES = {
    "kcore_create": ([ctypes.POINTER(c_p), ctypes.c_int], ctypes.c_int),
    "kcore_destroy": ([c_p], ctypes.c_int),
    "kcore_last_error": ([c_p], ctypes.c_char_p),
    "kcore_set_option": ([c_p, ctypes.c_int, c_i64], ctypes.c_int),
    "kcore_get_option": ([c_p, ctypes.c_int, ctypes.POINTER(c_i64)], ctypes.c_int),
    "kcore_workspace_size": ([c_p, c_i64, c_i64, ctypes.POINTER(c_sz)], ctypes.c_int),
    "kcore_set_workspace": ([c_p, c_p, c_sz], ctypes.c_int),
    "kcore_decompose": ([c_p, c_i64, c_i64, c_p, c_p, c_p, c_p, c_p], ctypes.c_int),
    "kcore_decompose_host": ([c_p, c_i64, c_i64, c_p, c_p, c_p, c_p, c_p], ctypes.c_int),
    "kcore_core_mask": ([c_p, c_i64, c_i64, c_p, c_p, ctypes.c_int32, c_p, c_p, c_p], ctypes.c_int),
    "kcore_validate_csr": ([c_p, c_i64, c_i64, c_p, c_p, c_p], ctypes.c_int),
    "kcore_sync_status": ([c_p], ctypes.c_int),
    "kcore_get_stats": ([c_p, ctypes.POINTER(Stats)], ctypes.c_int),
    "kcore_barrier_latency": ([c_p, c_i64, ctypes.c_int32, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    "kcore_get_trace": ([c_p, c_p, c_i64, ctypes.POINTER(c_i64)], ctypes.c_int),
    "kcore_build_csr": ([c_p, c_i64, c_i64, c_p, c_p, c_p, c_p, c_p, c_p], ctypes.c_int),
    "kcore_build_csr_workspace_size": ([c_p, c_i64, c_i64, ctypes.POINTER(c_sz)], ctypes.c_int),
    "kcore_decompose_static": ([c_i64, c_i64, c_p, c_p, c_p, c_p, c_p], ctypes.c_int),
    "kcore_decompose_batched": ([c_p, c_i64, c_i64, c_i64, c_p, c_p, c_p, c_p, c_p, c_p],
                                ctypes.c_int),
    "kcore_batched_workspace_size": ([c_p, c_i64, c_i64, ctypes.POINTER(c_sz)], ctypes.c_int),
    "kcore_autotune_batched": ([c_p, c_i64, c_i64, c_i64, c_p, c_p, c_p, c_p, c_p, ctypes.c_int32,
                                ctypes.POINTER(BatchTuning), c_p], ctypes.c_int),
    "kcore_autotune": ([c_p, c_i64, c_i64, c_p, c_p, c_p, c_p, ctypes.c_int32, ctypes.POINTER(Tuning), c_p],
                       ctypes.c_int),
    "kcore_build_csr_batched": ([c_p, c_i64, c_i64, c_i64, c_i64, c_p, c_p, c_p, c_p, c_p, c_p, c_p,
                                 c_p], ctypes.c_int),
    "kcore_server_create": ([ctypes.POINTER(c_p), ctypes.c_int, c_p], ctypes.c_int),
    "kcore_server_submit": ([c_p, c_i64, c_i64, c_p, c_p, c_p, ctypes.POINTER(c_i64)], ctypes.c_int),
    "kcore_server_poll": ([c_p, c_p, c_p, c_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)], ctypes.c_int),
    "kcore_server_info": ([c_p, ctypes.POINTER(c_i64), ctypes.POINTER(c_i64), ctypes.POINTER(c_i64)],
                          ctypes.c_int),
    "kcore_server_destroy": ([c_p], ctypes.c_int),
}


class ServerConfig(ctypes.Structure):
    _fields_ = [("pool_bytes", c_sz), ("max_requests", ctypes.c_int), ("streams", ctypes.c_int),
                ("large_vertices", c_i64), ("large_arcs", c_i64), ("batch_cluster", ctypes.c_int),
                ("batch_big_arcs", c_i64)]


def _declare(L):
    for name, (args, res) in SIGNATURES.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
