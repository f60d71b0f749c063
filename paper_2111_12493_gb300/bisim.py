"""Python binding of libbisim_gb300 (include/bisim.h): argument marshalling only.

Every function has the name of the C entry point it calls. Arrays are torch
tensors, on the current CUDA device or in (preferably pinned) host memory;
their data pointers go to the library unchanged, and all computation runs in
the library's CUDA kernels. There is no fallback: if the shared library is
missing or fails to load, importing this module raises.
"""

from __future__ import annotations

import ctypes
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbisim_gb300.so")

FIXPOINT = -1
FLAG_L2_PIN, FLAG_FULL_RECOMPUTE, FLAG_EAGER, FLAG_UNION_ROUNDS = 1, 2, 4, 8
DIR_FORWARD, DIR_BACKWARD, DIR_BOTH = 0, 1, 2
OP_EDGE_ADD, OP_EDGE_DEL, OP_VERTEX_ADD, OP_VERTEX_DEL = 0, 1, 2, 3

_STATUS = {0: "BISIM_OK", 1: "BISIM_EINVAL", 2: "BISIM_ENOMEM", 3: "BISIM_ECUDA",
           4: "BISIM_ESTATE", 5: "BISIM_ETIMEOUT", 6: "BISIM_EADMIT"}


class BisimError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status
        self.message = message


class Options(ctypes.Structure):
    _fields_ = [("k_incremental", ctypes.c_int32), ("hash_bits", ctypes.c_int32),
                ("small_max_degree", ctypes.c_int32), ("mid_max_degree", ctypes.c_int32),
                ("hub_chunk", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("mem_budget_bytes", ctypes.c_int64), ("direction", ctypes.c_int32),
                ("n_label_filter", ctypes.c_int32), ("label_filter", ctypes.c_void_p),
                ("batch_split", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("n_vertices", ctypes.c_int32), ("n_graphs", ctypes.c_int32), ("n_edges", ctypes.c_int64),
                ("rounds", ctypes.c_int32), ("rounds_executed", ctypes.c_int32),
                ("num_blocks", ctypes.c_int64), ("collision_levels", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("n_small", ctypes.c_int64), ("n_mid", ctypes.c_int64),
                ("n_hub", ctypes.c_int64), ("updates_applied", ctypes.c_int64),
                ("last_frontier", ctypes.c_int64), ("state_builds", ctypes.c_int64)]


class KernelProfile(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 40), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double),
                ("alg_bytes", ctypes.c_double), ("vertices", ctypes.c_int64), ("edges", ctypes.c_int64)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing; build it with paper_2111_12493_gb300.build.build()")
    lib = ctypes.CDLL(LIB_PATH)
    p, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
    pp = ctypes.POINTER(ctypes.c_void_p)
    sigs = {
        "bisim_default_options": (None, [ctypes.POINTER(Options)]),
        "summarize_init": (ctypes.c_int, [pp, i32, i64, p, p, p, p, p, ctypes.POINTER(Options), p]),
        "summarize_init_coo": (ctypes.c_int, [pp, i32, i64, p, p, p, p, p, ctypes.POINTER(Options), p]),
        "summarize_init_batched": (ctypes.c_int, [pp, i32, p, p, p, p, p, p, ctypes.POINTER(Options), p]),
        "bisim_iterate": (ctypes.c_int, [p, i32, i32, ctypes.POINTER(i32), ctypes.POINTER(i64), p]),
        "apply_updates": (ctypes.c_int, [p, p, i64, p]),
        "get_partition": (ctypes.c_int, [p, p, p]),
        "bisim_get_stats": (ctypes.c_int, [p, ctypes.POINTER(Stats)]),
        "summarize_destroy": (ctypes.c_int, [p]),
        "bisim_last_error": (ctypes.c_char_p, [p]),
        "bisim_profile_enable": (None, [i32]),
        "bisim_profile_reset": (None, []),
        "bisim_profile_read": (i32, [ctypes.POINTER(KernelProfile), i32]),
        "bisim_launch_count": (i64, []),
        "bisim_refine_round_noalloc": (ctypes.c_int, [i32, i64, p, p, p, p, p, ctypes.POINTER(i64), p]),
        "bisim_autotune": (ctypes.c_int, [p, i32, ctypes.POINTER(Options), p]),
        "bisim_retune": (ctypes.c_int, [p, ctypes.POINTER(Options), p]),
        "get_block_sizes": (ctypes.c_int, [p, p, p]),
        "bisim_literal_alg4": (ctypes.c_int, [p, i32, p, ctypes.POINTER(i64), p]),
        "bisim_export_state": (ctypes.c_int, [p, p, i64, ctypes.POINTER(i64), p]),
        "bisim_import_state": (ctypes.c_int, [pp, p, i64, p]),
        "get_summary_edges": (ctypes.c_int, [p, p, p, p, i64, ctypes.POINTER(i64), p]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()


def default_options(**overrides) -> Options:
    """bisim_default_options with fields overridden; `label_filter` takes a
    sequence of edge labels (kept alive with the options)."""
    o = Options()
    _lib.bisim_default_options(ctypes.byref(o))
    labels = overrides.pop("label_filter", None)
    for k, v in overrides.items():
        setattr(o, k, v)
    if labels is not None:
        arr = (ctypes.c_int32 * max(1, len(labels)))(*[int(x) for x in labels])
        o._label_filter_keep = arr
        o.n_label_filter = len(labels)
        o.label_filter = ctypes.cast(arr, ctypes.c_void_p)
    return o


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t, dtype, name, n=None):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor):
        raise TypeError(f"{name} must be a torch.Tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if n is not None and t.numel() != n:
        raise ValueError(f"{name} must have {n} elements, got {t.numel()}")
    return ctypes.c_void_p(t.data_ptr()) if t.numel() > 0 else None


def _check(rc, ctx_ptr=None):
    if rc != 0:
        msg = _lib.bisim_last_error(ctx_ptr)
        raise BisimError(rc, msg.decode() if msg else "")


class Context:
    """An owned bisim_ctx; freed by summarize_destroy (or when collected)."""

    def __init__(self, ptr, n_vertices, batched=False):
        self._ptr = ptr
        self.n_vertices = n_vertices
        self.batched = batched
        self._keep = None

    @property
    def ptr(self):
        if self._ptr is None:
            raise ValueError("context already destroyed")
        return self._ptr

    def __del__(self):
        if getattr(self, "_ptr", None) is not None:
            _lib.summarize_destroy(self._ptr)
            self._ptr = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        summarize_destroy(self)


def summarize_init(n_vertices, row_ptr, col, edge_label, vertex_label, alive=None, options=None,
                   stream=None) -> Context:
    out = ctypes.c_void_p()
    m = col.numel()
    rc = _lib.summarize_init(ctypes.byref(out), n_vertices, m, _ptr(row_ptr, torch.int64, "row_ptr", n_vertices + 1),
                             _ptr(col, torch.int32, "col"), _ptr(edge_label, torch.int32, "edge_label", m),
                             _ptr(vertex_label, torch.int32, "vertex_label", n_vertices),
                             _ptr(alive, torch.uint8, "alive", n_vertices),
                             ctypes.byref(options) if options is not None else None, _stream(stream))
    _check(rc)
    return Context(out, n_vertices)


def summarize_init_coo(n_vertices, src, dst, edge_label, vertex_label, alive=None, options=None,
                       stream=None) -> Context:
    out = ctypes.c_void_p()
    m = src.numel()
    rc = _lib.summarize_init_coo(ctypes.byref(out), n_vertices, m, _ptr(src, torch.int32, "src"),
                                 _ptr(dst, torch.int32, "dst", m), _ptr(edge_label, torch.int32, "edge_label", m),
                                 _ptr(vertex_label, torch.int32, "vertex_label", n_vertices),
                                 _ptr(alive, torch.uint8, "alive", n_vertices),
                                 ctypes.byref(options) if options is not None else None, _stream(stream))
    _check(rc)
    return Context(out, n_vertices)


def summarize_init_batched(vertex_offsets, edge_offsets, src_local, dst_local, edge_label, vertex_label,
                           options=None, stream=None) -> Context:
    out = ctypes.c_void_p()
    g = vertex_offsets.numel() - 1
    rc = _lib.summarize_init_batched(ctypes.byref(out), g, _ptr(vertex_offsets, torch.int64, "vertex_offsets"),
                                     _ptr(edge_offsets, torch.int64, "edge_offsets", g + 1),
                                     _ptr(src_local, torch.int32, "src_local"),
                                     _ptr(dst_local, torch.int32, "dst_local", src_local.numel()),
                                     _ptr(edge_label, torch.int32, "edge_label", src_local.numel()),
                                     _ptr(vertex_label, torch.int32, "vertex_label"),
                                     ctypes.byref(options) if options is not None else None, _stream(stream))
    _check(rc)
    return Context(out, vertex_label.numel(), batched=True)


def bisim_iterate(ctx: Context, k: int, cap: int = 10, stream=None):
    """Returns (rounds, num_blocks)."""
    rounds = ctypes.c_int32()
    blocks = ctypes.c_int64()
    rc = _lib.bisim_iterate(ctx.ptr, k, cap, ctypes.byref(rounds), ctypes.byref(blocks), _stream(stream))
    _check(rc, ctx.ptr)
    return rounds.value, blocks.value


def apply_updates(ctx: Context, ops, stream=None):
    """ops: int32 tensor [n_ops, 4] of rows (kind, src, dst, label)."""
    if ops.dim() != 2 or ops.shape[1] != 4:
        raise ValueError("ops must have shape [n_ops, 4]")
    rc = _lib.apply_updates(ctx.ptr, _ptr(ops, torch.int32, "ops"), ops.shape[0], _stream(stream))
    _check(rc, ctx.ptr)


def get_partition(ctx: Context, out=None, stream=None):
    if out is None:
        out = torch.empty(ctx.n_vertices, dtype=torch.int32, device="cuda")
    rc = _lib.get_partition(ctx.ptr, _ptr(out, torch.int32, "out", ctx.n_vertices), _stream(stream))
    _check(rc, ctx.ptr)
    return out


def get_block_sizes(ctx: Context, out=None, stream=None):
    """Vertices per block: out[b] = |{v : P[v] = b}| (0 where b is not a block id)."""
    if out is None:
        out = torch.empty(ctx.n_vertices, dtype=torch.int32, device="cuda")
    _check(_lib.get_block_sizes(ctx.ptr, _ptr(out, torch.int32, "out", ctx.n_vertices), _stream(stream)), ctx.ptr)
    return out


def get_summary_edges(ctx: Context, stream=None):
    """The summary graph's edges as three int32 device tensors (source block,
    label, target block), distinct and sorted lexicographically."""
    count = ctypes.c_int64()
    cap = max(1, int(bisim_get_stats(ctx)["n_edges"]))
    while True:
        outs = [torch.empty(cap, dtype=torch.int32, device="cuda") for _ in range(3)]
        _check(_lib.get_summary_edges(ctx.ptr, *[ctypes.c_void_p(o.data_ptr()) for o in outs], cap,
                                      ctypes.byref(count), _stream(stream)), ctx.ptr)
        if count.value <= cap:
            return tuple(o[:count.value] for o in outs)
        cap = count.value


def bisim_export_state(ctx: Context, stream=None) -> bytes:
    """The context's state (graph, options, partition, incremental levels) as bytes."""
    size = ctypes.c_int64()
    _check(_lib.bisim_export_state(ctx.ptr, None, 0, ctypes.byref(size), _stream(stream)), ctx.ptr)
    buf = ctypes.create_string_buffer(size.value)
    _check(_lib.bisim_export_state(ctx.ptr, buf, size.value, ctypes.byref(size), _stream(stream)), ctx.ptr)
    return buf.raw


def bisim_import_state(blob: bytes, stream=None) -> Context:
    """A new context from bisim_export_state's bytes."""
    out = ctypes.c_void_p()
    buf = ctypes.create_string_buffer(blob, len(blob))
    _check(_lib.bisim_import_state(ctypes.byref(out), buf, len(blob), _stream(stream)))
    n = ctypes.cast(buf, ctypes.POINTER(ctypes.c_int32))[4]      # StateHeader.n follows magic, version, size
    return Context(out, n)


def bisim_literal_alg4(ctx: Context, k: int, out=None, stream=None):
    """Diagnostic: the partition of Algorithm 4 taken literally (two identifier
    tracks, no edge labels in the last round). Returns (partition, blocks)."""
    if out is None:
        out = torch.empty(ctx.n_vertices, dtype=torch.int32, device="cuda")
    blocks = ctypes.c_int64()
    _check(_lib.bisim_literal_alg4(ctx.ptr, k, _ptr(out, torch.int32, "out", ctx.n_vertices), ctypes.byref(blocks),
                                   _stream(stream)), ctx.ptr)
    return out, blocks.value


def bisim_autotune(ctx: Context, rounds: int = 2, stream=None) -> dict:
    """Time candidate class thresholds and hub chunk sizes on this graph; keep the fastest.

    Returns the chosen options as a dict; they apply from the next
    bisim_iterate (the current partition is left undefined until then).
    """
    o = Options()
    _check(_lib.bisim_autotune(ctx.ptr, rounds, ctypes.byref(o), _stream(stream)), ctx.ptr)
    return {name: getattr(o, name) for name, _ in Options._fields_}


TUNING_FIELDS = ("small_max_degree", "mid_max_degree", "hub_chunk", "batch_split")


def bisim_retune(ctx: Context, stream=None, **settings) -> None:
    """Set the context's tuning options (TUNING_FIELDS) without timing; the
    layout is rebuilt by the next bisim_iterate or apply_updates."""
    unknown = set(settings) - set(TUNING_FIELDS)
    if unknown:
        raise ValueError(f"not tuning options: {sorted(unknown)}")
    o = default_options(**settings)
    _check(_lib.bisim_retune(ctx.ptr, ctypes.byref(o), _stream(stream)), ctx.ptr)


def bisim_get_stats(ctx: Context) -> dict:
    s = Stats()
    _check(_lib.bisim_get_stats(ctx.ptr, ctypes.byref(s)), ctx.ptr)
    return {name: getattr(s, name) for name, _ in Stats._fields_}


def summarize_destroy(ctx: Context):
    if ctx._ptr is not None:
        _lib.summarize_destroy(ctx._ptr)
        ctx._ptr = None


def bisim_last_error(ctx: Context | None = None) -> str:
    msg = _lib.bisim_last_error(ctx.ptr if ctx is not None else None)
    return msg.decode() if msg else ""


def bisim_profile_enable(enable: bool = True):
    _lib.bisim_profile_enable(1 if enable else 0)


def bisim_profile_reset():
    _lib.bisim_profile_reset()


def bisim_profile_read() -> list:
    """Per launch site: name, launches, total_ms, alg_bytes, vertices, edges."""
    n = _lib.bisim_profile_read(None, 0)
    arr = (KernelProfile * max(n, 1))()
    n = _lib.bisim_profile_read(arr, n)
    return [dict(name=a.name.decode(), launches=a.launches, total_ms=a.total_ms, alg_bytes=a.alg_bytes,
                 vertices=a.vertices, edges=a.edges) for a in arr[:n]]


def bisim_launch_count() -> int:
    return int(_lib.bisim_launch_count())


def bisim_refine_round_noalloc(n_vertices, row_ptr, col, edge_label, block_in, block_out, stream=None) -> int:
    """One refinement round into caller-provided block_out without any allocation.

    For callers that may not allocate device memory (a plugin inside another
    runtime that owns the device heap, a loop that reserves all buffers up
    front); scratch comes from a fixed array inside the library. All tensors
    must be on the device; returns the number of blocks of block_out.
    """
    blocks = ctypes.c_int64()
    m = col.numel()
    rc = _lib.bisim_refine_round_noalloc(n_vertices, m, _ptr(row_ptr, torch.int64, "row_ptr", n_vertices + 1),
                                         _ptr(col, torch.int32, "col"), _ptr(edge_label, torch.int32, "edge_label", m),
                                         _ptr(block_in, torch.int32, "block_in", n_vertices),
                                         _ptr(block_out, torch.int32, "block_out", n_vertices),
                                         ctypes.byref(blocks), _stream(stream))
    _check(rc)
    return blocks.value
