"""C ABI checks that need no GPU: the library builds for sm_103a, loads, and
exports every entry point include/kcore.h declares; host-side argument
validation answers without touching a device."""
import ctypes
import os
import re

from paper_2502_08042_gb300 import _native

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not hdr.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", hdr)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?\w+\s*\*?\s+(kcore_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return names


def test_header_declares_entry_points():
    names = declared_functions()
    for required in ("kcore_create", "kcore_decompose", "kcore_destroy", "kcore_sync_status"):
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = _native.lib()
    for name in sorted(declared_functions()):
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"


def test_binding_covers_every_declared_symbol():
    assert declared_functions() <= set(_native.SIGNATURES)


def test_argument_errors_without_device():
    lib = _native.lib()
    assert lib.kcore_create(None, 0) == 1  # KCORE_ERR_INVALID
    assert lib.kcore_last_error(None) == b"null handle"
    assert lib.kcore_decompose(None, 0, 0, None, None, None, None, None) == 1
    assert lib.kcore_sync_status(None) == 1
    assert lib.kcore_destroy(None) == 1


def test_build_targets_sm103a_only():
    assert _native.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_smoke_graph_is_well_formed():
    """The input smoke() sends to the GPU builds on the CPU and holds the
    staircase's top level."""
    import __graft_entry__ as ge
    import oracle
    n, s, d = ge.smoke_graph()
    off, adj = oracle.build_csr(n, s, d)
    assert len(off) == n + 1 and oracle.check_simple(n, off, adj) == 0
    assert int(oracle.bz(n, off, adj).max()) >= 40
