"""The C-ABI library loads without a GPU and exports every entry point of include/bisim.h."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bisim.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^(?:bisim_status|void|const char\*)\s+(\w+)\s*\(", text, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("summarize_init", "summarize_init_coo", "summarize_init_batched", "bisim_iterate",
                     "apply_updates", "get_partition", "summarize_destroy", "bisim_last_error"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_2111_12493_gb300 import build
    try:
        path = build.build()
    except RuntimeError as e:  # no CUDA toolkit on this machine
        pytest.skip(str(e))
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_default_options_without_gpu():
    from paper_2111_12493_gb300 import build
    try:
        path = build.build()
    except RuntimeError as e:
        pytest.skip(str(e))
    lib = ctypes.CDLL(path)

    # the whole bisim_options of include/bisim.h: the call writes every field
    class Options(ctypes.Structure):
        _fields_ = [("k_incremental", ctypes.c_int32), ("hash_bits", ctypes.c_int32),
                    ("small_max_degree", ctypes.c_int32), ("mid_max_degree", ctypes.c_int32),
                    ("hub_chunk", ctypes.c_int32), ("flags", ctypes.c_int32),
                    ("mem_budget_bytes", ctypes.c_int64), ("direction", ctypes.c_int32),
                    ("n_label_filter", ctypes.c_int32), ("label_filter", ctypes.c_void_p),
                    ("batch_split", ctypes.c_int32)]

    class Guarded(ctypes.Structure):
        _fields_ = [("o", Options), ("guard", ctypes.c_uint8 * 64)]

    g = Guarded()
    ctypes.memset(g.guard, 0xA5, 64)
    lib.bisim_default_options(ctypes.byref(g.o))
    o = g.o
    assert (o.k_incremental, o.hash_bits, o.small_max_degree, o.mid_max_degree) == (2, 64, 32, 8192)
    assert (o.hub_chunk, o.flags, o.mem_budget_bytes, o.direction, o.n_label_filter) == (4096, 0, 0, 0, 0)
    assert not o.label_filter and o.batch_split >= 0
    assert bytes(g.guard) == b"\xa5" * 64, "bisim_default_options wrote past the struct this test declares"
    lib.bisim_last_error.restype = ctypes.c_char_p
    assert lib.bisim_last_error(None) is not None


def test_calls_fail_loudly_without_a_gpu():
    """No CPU fallback: without a device every call returns an error status (and the binding raises)."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import numpy as np
    from paper_2111_12493_gb300 import build
    try:
        path = build.build()
    except RuntimeError as e:
        pytest.skip(str(e))
    lib = ctypes.CDLL(path)
    lib.bisim_last_error.restype = ctypes.c_char_p
    out = ctypes.c_void_p()
    vl = np.zeros(2, np.int32)
    rc = lib.summarize_init_coo(ctypes.byref(out), 2, ctypes.c_int64(0), None, None, None,
                                vl.ctypes.data_as(ctypes.c_void_p), None, None, None)
    assert rc == 3 and out.value is None           # BISIM_ECUDA, no context
    assert lib.bisim_last_error(None)
    from paper_2111_12493_gb300 import bisim
    with pytest.raises(RuntimeError):
        bisim.summarize_init_coo(2, torch.zeros(0, dtype=torch.int32), torch.zeros(0, dtype=torch.int32),
                                 torch.zeros(0, dtype=torch.int32), torch.zeros(2, dtype=torch.int32))


def _header_struct(name):
    """Fields of `typedef struct { ... } name;` in the header as (field, kind)
    pairs, kind one of i32, i64, f64, ptr, char[N]."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    m = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + r"\s*;", text)
    assert m, name
    fields = []
    for decl in m.group(1).split(";"):
        decl = " ".join(decl.split())
        if not decl:
            continue
        arr = re.fullmatch(r"char (\w+)\[(\d+)\]", decl)
        if arr:
            fields.append((arr.group(1), f"char[{arr.group(2)}]"))
            continue
        typ, names = re.fullmatch(r"((?:const )?\w+\s*\*?)\s*(.+)", decl).groups()
        kind = "ptr" if "*" in typ else {"int32_t": "i32", "int64_t": "i64", "double": "f64"}[typ.strip()]
        fields.extend((n.strip(), kind) for n in names.split(","))
    return fields


def _ctypes_kind(t):
    import ctypes as C
    if t is C.c_int32:
        return "i32"
    if t is C.c_int64:
        return "i64"
    if t is C.c_double:
        return "f64"
    if t is C.c_void_p:
        return "ptr"
    if issubclass(t, C.Array) and t._type_ is C.c_char:
        return f"char[{t._length_}]"
    raise AssertionError(t)


@pytest.mark.parametrize("cname,pyname", [("bisim_options", "Options"), ("bisim_stats", "Stats"),
                                          ("bisim_kernel_profile", "KernelProfile")])
def test_binding_structs_mirror_the_header(cname, pyname):
    # the ctypes mirrors of the binding must match the header field by field,
    # or calls would read and write past them
    try:
        from paper_2111_12493_gb300 import bisim
    except (OSError, RuntimeError) as e:  # library not built here
        pytest.skip(str(e))
    py = [(f, _ctypes_kind(t)) for f, t in getattr(bisim, pyname)._fields_]
    assert py == _header_struct(cname)


def test_update_rows_match_the_op_struct():
    # apply_updates takes [n_ops, 4] int32 rows (kind, src, dst, label): bisim_op
    # must be exactly those four 32-bit fields, in that order
    assert _header_struct("bisim_op") == [("kind", "i32"), ("src", "i32"), ("dst", "i32"), ("label", "i32")]
