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


def _header_text():
    text = open(os.path.join(ROOT, "include", "kcore.h")).read()
    return re.sub(r"/\*.*?\*/", "", text, flags=re.S)


def test_binding_option_names_match_the_header():
    """Every KCORE_OPT_* of the header has the binding's name and value, and
    the binding names no option the header lacks."""
    from paper_2502_08042_gb300 import kcore
    enum = re.search(r"typedef enum\s*\{(.*?)\}\s*kcore_option\s*;", _header_text(), flags=re.S).group(1)
    opts = {m.group(1).lower(): int(m.group(2)) for m in re.finditer(r"KCORE_OPT_(\w+)\s*=\s*(\d+)", enum)}
    assert opts == kcore.OPTIONS
    assert sorted(opts.values()) == list(range(len(opts)))  # dense, no gaps


def test_stats_struct_matches_the_header():
    """The binding's kcore_stats mirror has the header's fields in order, all
    int64, so ctypes reads the same bytes the library writes."""
    body = re.search(r"typedef struct\s*\{([^{}]*)\}\s*kcore_stats\s*;", _header_text()).group(1)
    fields = re.findall(r"int64_t\s+(\w+)\s*;", body)
    assert [name for name, _ in _native.Stats._fields_] == fields
    assert ctypes.sizeof(_native.Stats) == 8 * len(fields)


def test_status_codes_match_the_header():
    from paper_2502_08042_gb300 import kcore
    enum = re.search(r"typedef enum\s*\{(.*?)\}\s*kcore_status\s*;", _header_text(), flags=re.S).group(1)
    codes = {int(m.group(2)): m.group(1) for m in re.finditer(r"KCORE_(?:ERR_)?(\w+)\s*=\s*(\d+)", enum)}
    for value, name in codes.items():
        assert kcore.STATUS[value].upper() == name, (value, name)


_CTYPES = {"int64_t": ctypes.c_int64, "int32_t": ctypes.c_int32, "int": ctypes.c_int, "size_t": ctypes.c_size_t,
           "double": ctypes.c_double}


def _struct_fields(name):
    body = re.search(r"typedef struct\s*\{([^{}]*)\}\s*" + name + r"\s*;", _header_text()).group(1)
    return [(m.group(2), m.group(1)) for m in re.finditer(r"(int64_t|int32_t|int|size_t|double)\s+(\w+)\s*;", body)]


def test_other_mirrored_structs_match_the_header():
    for cname, mirror in (("kcore_batch_tuning", _native.BatchTuning), ("kcore_server_config", _native.ServerConfig),
                          ("kcore_tuning", _native.Tuning)):
        fields = _struct_fields(cname)
        assert [n for n, _ in mirror._fields_] == [n for n, _ in fields], cname
        for (n, ct), (_, cty) in zip(mirror._fields_, fields):
            assert ctypes.sizeof(ct) == ctypes.sizeof(_CTYPES[cty]), (cname, n)
