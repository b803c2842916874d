"""Thin Python binding of libms (include/morphstore.h) over ctypes.

Argument marshalling only: every step of every operator runs in libms's CUDA
kernels.  PyTorch supplies device memory (the caching allocator backs the
library's allocator callbacks), tensors for caller-owned buffers and the current
stream.  The binding refuses to load without the compiled library: there is no
fallback path.
"""
from __future__ import annotations

import ctypes
import os
import re
import weakref

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_PKG, "libms.so")
_HEADER = os.path.join(os.path.dirname(_PKG), "include", "morphstore.h")

UNCOMPR, STATIC_BP, DYN_BP, DELTA_BP, FOR_BP, RLE, FOR_STATIC_BP, DELTA_STATIC_BP = range(8)
FORMAT_NAMES = ("uncompr", "static_bp", "dyn_bp", "delta_bp", "for_bp", "rle", "for_static_bp", "delta_static_bp")
EQ, NE, LT, LE, GT, GE, BETWEEN = range(7)
ADD, SUB, MUL = range(3)
STATUS = ("MS_OK", "MS_ERR_INVALID_ARG", "MS_ERR_FORMAT", "MS_ERR_VALUE_TOO_WIDE",
          "MS_ERR_OUT_OF_RANGE", "MS_ERR_NOMEM", "MS_ERR_TIMEOUT", "MS_ERR_CUDA")
(MS_OK, MS_ERR_INVALID_ARG, MS_ERR_FORMAT, MS_ERR_VALUE_TOO_WIDE, MS_ERR_OUT_OF_RANGE,
 MS_ERR_NOMEM, MS_ERR_TIMEOUT, MS_ERR_CUDA) = range(8)


class MSError(RuntimeError):
    def __init__(self, code: int, what: str, info: int = 0):
        name = STATUS[code] if 0 <= code < len(STATUS) else str(code)
        super().__init__(f"{what}: {name} (info {info})")
        self.code = code
        self.info = info


class KernelTime(ctypes.Structure):
    _fields_ = [("kernel", ctypes.c_int32), ("launches", ctypes.c_uint32), ("total_ms", ctypes.c_double)]


class BatchConfig(ctypes.Structure):
    """ms_batch_config: warps per CTA, chunks in flight per warp, chunks per tile
    (power of two), CTAs per SM (0 = as many as fit), compact decoder flag,
    schedule (0 = tiles to warps from a work counter, 1 = tiles round-robin to CTAs,
    2 = runs of chunks streamed through CTA-wide shared-memory buffers)."""
    _fields_ = [("warps", ctypes.c_uint32), ("depth", ctypes.c_uint32), ("tile_chunks", ctypes.c_uint32),
                ("ctas_per_sm", ctypes.c_uint32), ("compact", ctypes.c_uint32), ("schedule", ctypes.c_uint32)]

    def as_tuple(self):
        return (self.warps, self.depth, self.tile_chunks, self.ctas_per_sm, self.compact, self.schedule)

    def __repr__(self):
        return ("BatchConfig(warps=%d, depth=%d, tile_chunks=%d, ctas_per_sm=%d, compact=%d, schedule=%d)"
                % self.as_tuple())


DEFAULT_BATCH_CONFIG = (8, 2, 32, 0, 0, 1)
# (warps, depth, compact, schedule) combinations the library is built with
# (schedule 2 streams runs of chunks through CTA-wide buffers of 8 KB x depth per column)
BATCH_VARIANTS = tuple([(w, d, c, 0) for w in (4, 8) for d in (2, 3, 4) for c in (0, 1)] +
                       [(4, 2, 0, 1), (8, 2, 0, 1), (16, 2, 0, 1), (4, 3, 0, 1), (8, 3, 0, 1)] +
                       [(8, 2, 0, 2), (8, 3, 0, 2), (8, 4, 0, 2)])
BATCH_ZERO, BATCH_PER_FRAGMENT = 1, 2


class ColumnMeta(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("fmt", ctypes.c_int32), ("static_bw", ctypes.c_int32),
                ("size_bytes", ctypes.c_uint64), ("n_blocks", ctypes.c_uint64),
                ("payload_words", ctypes.c_uint64), ("device_ptr", ctypes.c_uint64)]


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)

_lib = None


def library_path() -> str:
    return _LIB_PATH


def load() -> ctypes.CDLL:
    """Loads libms.so; raises if it has not been built (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(f"libms.so is missing at {_LIB_PATH}; run __graft_entry__.build() first")
    lib = ctypes.CDLL(_LIB_PATH)
    p, u64, i32 = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int
    pp = ctypes.POINTER(ctypes.c_void_p)
    sigs = {
        "ms_ctx_create": [pp, i32, u64, u64, _ALLOC_FN, _FREE_FN, p],
        "ms_ctx_destroy": [p],
        "ms_get_error": [p, p],
        "ms_arena_usage": [p, ctypes.POINTER(u64), ctypes.POINTER(u64), p],
        "ms_arena_reset_high_water": [p, p],
        "ms_column_import": [p, i32, i32, u64, p, u64, pp, p],
        "ms_column_export": [p, p, p, u64, ctypes.POINTER(u64), p],
        "ms_column_info": [p, p, ctypes.POINTER(ColumnMeta), p],
        "ms_column_free": [p, p, p],
        "ms_compress": [p, p, u64, i32, i32, pp, p],
        "ms_decompress": [p, p, p, u64, p],
        "ms_morph": [p, p, i32, i32, pp, p],
        "ms_select": [p, p, i32, u64, u64, i32, i32, pp, p],
        "ms_select_packed": [p, p, i32, u64, u64, i32, i32, pp, p],
        "ms_project": [p, p, p, i32, i32, pp, p],
        "ms_calc": [p, i32, p, p, u64, i32, i32, pp, p],
        "ms_agg_sum": [p, p, p, p],
        "ms_group_sum": [p, p, p, u64, p, p],
        "ms_semijoin": [p, p, p, u64, i32, i32, pp, p],
        "ms_compress_noalloc": [p, u64, i32, i32, p, u64, p, p],
        "ms_column_stats": [p, p, p, p],
        "ms_mlp_forward": [p, p, u64, p, p],
        "ms_mlp_loss_grad": [p, p, p, p, u64, ctypes.c_float, p, p, p, u64, p],
        "ms_mlp_adam": [p, p, p, p, u64, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, p],
    }
    sigs.update({
        "ms_batch_create": [p, ctypes.c_uint32, p, p, p, p, p, pp, p],
        "ms_batch_info": [p, ctypes.POINTER(u64), ctypes.POINTER(u64), ctypes.POINTER(u64)],
        "ms_batch_run": [p, ctypes.c_uint32, ctypes.c_uint32, ctypes.POINTER(BatchConfig), ctypes.c_uint32, p, p],
        "ms_batch_graph": [p, ctypes.c_uint32, ctypes.c_uint32, ctypes.POINTER(BatchConfig), ctypes.c_uint32, p, pp],
        "ms_graph_launch": [p, p],
        "ms_graph_destroy": [p],
        "ms_batch_destroy": [p],
        "ms_selftest_wait_timeout": [p, p],
    })
    for name, args in sigs.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.ms_profile_enable.argtypes = [p, i32]
    lib.ms_profile_enable.restype = ctypes.c_int
    lib.ms_profile_collect.argtypes = [p, ctypes.POINTER(KernelTime), i32, ctypes.POINTER(i32)]
    lib.ms_profile_collect.restype = ctypes.c_int
    lib.ms_kernel_name.argtypes = [i32]
    lib.ms_kernel_name.restype = ctypes.c_char_p
    lib.ms_last_cuda_error.argtypes = []
    lib.ms_last_cuda_error.restype = ctypes.c_int
    lib.ms_cuda_error_string.argtypes = [ctypes.c_int]
    lib.ms_cuda_error_string.restype = ctypes.c_char_p
    lib.ms_last_error_info.argtypes = [p]
    lib.ms_last_error_info.restype = u64
    lib.ms_column_max_rows.argtypes = [p]
    lib.ms_column_max_rows.restype = u64
    lib.ms_work_bytes.argtypes = [p]
    lib.ms_work_bytes.restype = u64
    _lib = lib
    return lib


def header_symbols() -> list[str]:
    """Names of the functions include/morphstore.h declares."""
    with open(_HEADER) as f:
        text = f.read()
    return sorted(set(re.findall(r"^\s*(?:ms_status|uint64_t|int|const char \*)\s*(ms_\w+)\s*\(", text, re.M)))


def _stream_handle(stream) -> ctypes.c_void_p:
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _check(code: int, what: str, ctx=None):
    if code != MS_OK:
        info = 0
        if ctx is not None:
            info = load().ms_last_error_info(ctx)
        if code == MS_ERR_CUDA:
            e = load().ms_last_cuda_error()
            what = f"{what} [cuda error {e}: {load().ms_cuda_error_string(e).decode()}]"
        raise MSError(code, what, info)


def as_device_u64(x, device) -> torch.Tensor:
    """uint64 numpy array (or int64 tensor) -> int64 CUDA tensor holding the same bits."""
    if isinstance(x, torch.Tensor):
        return x.to(device=device, dtype=torch.int64).contiguous()
    a = np.ascontiguousarray(np.asarray(x, dtype=np.uint64))
    return torch.from_numpy(a.view(np.int64)).to(device)


class Column:
    """Handle of a column owned by a context (opaque ms_column*)."""

    __slots__ = ("ctx", "ptr", "fmt", "bw")

    def __init__(self, ctx: "Ctx", ptr: int, fmt: int, bw: int):
        self.ctx, self.ptr, self.fmt, self.bw = ctx, ptr, fmt, bw

    @property
    def max_rows(self) -> int:
        return int(load().ms_column_max_rows(self.ptr))

    def info(self, stream=None) -> dict:
        return self.ctx.info(self, stream)

    def __repr__(self):
        return f"Column(fmt={FORMAT_NAMES[self.fmt]}, bw={self.bw}, max_rows={self.max_rows})"


class Ctx:
    """A libms context on one device (see ms_ctx_create)."""

    def __init__(self, device: int = 0, arena_bytes: int = 1 << 30, max_rows: int = 1 << 20,
                 torch_allocator: bool = True):
        lib = load()
        self.device = torch.device("cuda", device)
        self._blocks = {}
        if torch_allocator:
            def _alloc(size, user):
                try:
                    t = torch.empty(int(size), dtype=torch.uint8, device=self.device)
                except RuntimeError:
                    return None
                self._blocks[t.data_ptr()] = t
                return t.data_ptr()

            def _free(ptr, user):
                self._blocks.pop(int(ptr), None)

            self._alloc_cb, self._free_cb = _ALLOC_FN(_alloc), _FREE_FN(_free)
        else:
            self._alloc_cb, self._free_cb = _ALLOC_FN(0), _FREE_FN(0)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            _check(lib.ms_ctx_create(ctypes.byref(h), device, arena_bytes, max_rows,
                                     self._alloc_cb, self._free_cb, None), "ms_ctx_create")
        self.h = h
        self.arena_bytes = arena_bytes

    # -------------------------------------------------------------- lifecycle
    def close(self):
        if getattr(self, "h", None):
            for ref in getattr(self, "_batches", ()):
                b = ref()
                if b is not None:
                    b.close()
            load().ms_ctx_destroy(self.h)
            self.h = None
            self._blocks.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---------------------------------------------------------------- errors
    def get_error(self, stream=None) -> int:
        return load().ms_get_error(self.h, _stream_handle(stream))

    def last_error_info(self) -> int:
        return int(load().ms_last_error_info(self.h))

    def check(self, stream=None, what="device"):
        code = self.get_error(stream)
        if code != MS_OK:
            raise MSError(code, what, self.last_error_info())

    def arena_usage(self, stream=None):
        a, b = ctypes.c_uint64(), ctypes.c_uint64()
        _check(load().ms_arena_usage(self.h, ctypes.byref(a), ctypes.byref(b), _stream_handle(stream)),
               "ms_arena_usage")
        return a.value, b.value

    def work_bytes(self) -> int:
        """Bytes of the context's work area (ms_work_bytes)."""
        return int(load().ms_work_bytes(self.h))

    def reset_high_water(self, stream=None):
        _check(load().ms_arena_reset_high_water(self.h, _stream_handle(stream)), "reset_high_water")

    # ---------------------------------------------------------- statistics
    def selftest_wait_timeout(self, stream=None):
        """Run one device wait that nothing satisfies; it must give up with
        MS_ERR_TIMEOUT in the error word (read it with get_error)."""
        _check(load().ms_selftest_wait_timeout(self.h, _stream_handle(stream)), "ms_selftest_wait_timeout")

    def column_stats(self, col: Column, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """ms_column_stats into an int64 device tensor of STATS_WORDS words."""
        if out is None:
            out = torch.empty(STATS_WORDS, dtype=torch.int64, device=self.device)
        _check(load().ms_column_stats(self.h, col.ptr, ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)),
               "ms_column_stats")
        return out

    # ------------------------------------------------------------- profiling
    def profile(self, on: bool = True):
        _check(load().ms_profile_enable(self.h, 1 if on else 0), "ms_profile_enable")

    def profile_collect(self) -> dict:
        """{kernel name: (launches, total device ms)} since the last collect (synchronises)."""
        arr = (KernelTime * 32)()
        n = ctypes.c_int()
        _check(load().ms_profile_collect(self.h, arr, 32, ctypes.byref(n)), "ms_profile_collect")
        lib = load()
        return {lib.ms_kernel_name(arr[i].kernel).decode(): (arr[i].launches, arr[i].total_ms)
                for i in range(n.value)}

    # --------------------------------------------------------------- columns
    def _new(self, out: ctypes.c_void_p, fmt: int, bw: int) -> Column:
        return Column(self, out.value, fmt, bw if fmt == STATIC_BP else 0)

    def import_bytes(self, fmt: int, n: int, data, bw: int = 0, stream=None) -> Column:
        """Column from bytes in the documented layout (numpy uint8 or a uint8 tensor, host or device)."""
        if isinstance(data, torch.Tensor):
            src, size, keep = data.data_ptr(), data.numel() * data.element_size(), data
        else:
            keep = np.ascontiguousarray(np.asarray(data, dtype=np.uint8))
            src, size = keep.ctypes.data, keep.size
        out = ctypes.c_void_p()
        _check(load().ms_column_import(self.h, fmt, bw, n, ctypes.c_void_p(src), size, ctypes.byref(out),
                                       _stream_handle(stream)), "ms_column_import", self.h)
        if not isinstance(data, torch.Tensor):
            torch.cuda.current_stream(self.device).synchronize() if stream is None else stream.synchronize()
        del keep
        return self._new(out, fmt, bw)

    def export_bytes(self, col: Column, stream=None, device: bool = False, pinned: bool = False):
        """The column's bytes: a host numpy uint8 array, a uint8 tensor on the
        context's device (device=True) or a pinned host uint8 tensor (pinned=True)."""
        meta = self.info(col, stream)
        n = max(meta["size_bytes"], 1)
        if device or pinned:
            buf = torch.empty(n, dtype=torch.uint8, device=self.device) if device else \
                torch.empty(n, dtype=torch.uint8, pin_memory=True)
            ptr = buf.data_ptr()
        else:
            buf = np.zeros(n, dtype=np.uint8)
            ptr = buf.ctypes.data
        got = ctypes.c_uint64()
        _check(load().ms_column_export(self.h, col.ptr, ctypes.c_void_p(ptr), n, ctypes.byref(got),
                                       _stream_handle(stream)), "ms_column_export")
        return buf[: got.value]

    def info(self, col: Column, stream=None) -> dict:
        m = ColumnMeta()
        _check(load().ms_column_info(self.h, col.ptr, ctypes.byref(m), _stream_handle(stream)),
               "ms_column_info")
        return {k: getattr(m, k) for k, _ in ColumnMeta._fields_}

    def free(self, col: Column, stream=None):
        _check(load().ms_column_free(self.h, col.ptr, _stream_handle(stream)), "ms_column_free")
        col.ptr = None

    # ------------------------------------------------------------- operators
    def compress(self, d_in: torch.Tensor, fmt: int, bw: int = 0, stream=None) -> Column:
        assert d_in.is_cuda and d_in.element_size() == 8 and d_in.is_contiguous()
        out = ctypes.c_void_p()
        _check(load().ms_compress(self.h, ctypes.c_void_p(d_in.data_ptr()), d_in.numel(), fmt, bw,
                                  ctypes.byref(out), _stream_handle(stream)), "ms_compress")
        return self._new(out, fmt, bw)

    def decompress(self, col: Column, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        if out is None:
            n = self.info(col, stream)["n"]
            out = torch.empty(max(n, 1), dtype=torch.int64, device=self.device)[:n]
        _check(load().ms_decompress(self.h, col.ptr, ctypes.c_void_p(out.data_ptr()), out.numel(),
                                    _stream_handle(stream)), "ms_decompress")
        return out

    def select_packed(self, col: Column, cmp: int, c1: int, c2: int = 0, fmt: int = UNCOMPR, bw: int = 0,
                      stream=None) -> Column:
        """ms_select_packed: the specialized select on a packed (block or static BP) column."""
        out = ctypes.c_void_p()
        _check(load().ms_select_packed(self.h, col.ptr, cmp, c1, c2, fmt, bw, ctypes.byref(out),
                                       _stream_handle(stream)), "ms_select_packed")
        return self._new(out, fmt, bw)

    def morph(self, col: Column, fmt: int, bw: int = 0, stream=None) -> Column:
        """ms_morph: the column's values in another format, block by block in registers."""
        out = ctypes.c_void_p()
        _check(load().ms_morph(self.h, col.ptr, fmt, bw, ctypes.byref(out), _stream_handle(stream)), "ms_morph")
        return self._new(out, fmt, bw)

    def select(self, col: Column, cmp: int, c1: int, c2: int = 0, fmt: int = UNCOMPR, bw: int = 0,
               stream=None) -> Column:
        out = ctypes.c_void_p()
        _check(load().ms_select(self.h, col.ptr, cmp, c1, c2, fmt, bw, ctypes.byref(out),
                                _stream_handle(stream)), "ms_select")
        return self._new(out, fmt, bw)

    def project(self, data: Column, pos: Column, fmt: int = UNCOMPR, bw: int = 0, stream=None) -> Column:
        out = ctypes.c_void_p()
        _check(load().ms_project(self.h, data.ptr, pos.ptr, fmt, bw, ctypes.byref(out),
                                 _stream_handle(stream)), "ms_project")
        return self._new(out, fmt, bw)

    def calc(self, op: int, a: Column, b: Column | None = None, c: int = 0, fmt: int = UNCOMPR,
             bw: int = 0, stream=None) -> Column:
        out = ctypes.c_void_p()
        _check(load().ms_calc(self.h, op, a.ptr, None if b is None else b.ptr, c, fmt, bw,
                              ctypes.byref(out), _stream_handle(stream)), "ms_calc")
        return self._new(out, fmt, bw)

    def agg_sum(self, col: Column, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty(1, dtype=torch.int64, device=self.device)
        _check(load().ms_agg_sum(self.h, col.ptr, ctypes.c_void_p(out.data_ptr()), _stream_handle(stream)),
               "ms_agg_sum")
        return out

    def group_sum(self, gid: Column, val: Column, n_groups: int, out: torch.Tensor | None = None,
                  stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty(max(n_groups, 1), dtype=torch.int64, device=self.device)[:n_groups]
        _check(load().ms_group_sum(self.h, gid.ptr, val.ptr, n_groups, ctypes.c_void_p(out.data_ptr()),
                                   _stream_handle(stream)), "ms_group_sum")
        return out

    def semijoin(self, probe: Column, keys: Column, key_domain: int, fmt: int = UNCOMPR, bw: int = 0,
                 stream=None) -> Column:
        out = ctypes.c_void_p()
        _check(load().ms_semijoin(self.h, probe.ptr, keys.ptr, key_domain, fmt, bw, ctypes.byref(out),
                                  _stream_handle(stream)), "ms_semijoin")
        return self._new(out, fmt, bw)


NOALLOC_MAX_ROWS = 1 << 24
MLP_PARAMS = 5898
STATS_WORDS = 80


def _dp(t: torch.Tensor) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr())


def mlp_forward(params: torch.Tensor, x: torch.Tensor, out: torch.Tensor | None = None, stream=None):
    """ms_mlp_forward: y[n][10] = MLP(x[n][16]) on the device (fp32)."""
    n = x.shape[0]
    if out is None:
        out = torch.empty((n, 10), dtype=torch.float32, device=x.device)
    _check(load().ms_mlp_forward(_dp(params), _dp(x), n, _dp(out), _stream_handle(stream)), "ms_mlp_forward")
    return out


def mlp_loss_grad(params, x, y, mask, inv_count: float, grad, loss, partials, stream=None):
    """ms_mlp_loss_grad into the caller's grad (5898 floats), loss (1 float) and scratch."""
    _check(load().ms_mlp_loss_grad(_dp(params), _dp(x), _dp(y), _dp(mask), x.shape[0], float(inv_count),
                                   _dp(grad), _dp(loss), _dp(partials), partials.numel(), _stream_handle(stream)),
           "ms_mlp_loss_grad")


def mlp_adam(params, grad, m, v, step: int, lr=3e-3, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(load().ms_mlp_adam(_dp(params), _dp(grad), _dp(m), _dp(v), step, lr, beta1, beta2, eps,
                              _stream_handle(stream)), "ms_mlp_adam")


def compress_noalloc(d_in: torch.Tensor, fmt: int, d_out: torch.Tensor, d_result: torch.Tensor,
                     bw: int = 0, stream=None) -> None:
    """ms_compress_noalloc: compress into caller memory without any device allocation.

    d_out receives the column bytes; d_result (2 int64 words on the device) the size
    in bytes and the device status.  Calls that overlap on the GPU race on the
    library's fixed scratch array."""
    assert d_in.is_cuda and d_in.element_size() == 8 and d_in.is_contiguous()
    _check(load().ms_compress_noalloc(ctypes.c_void_p(d_in.data_ptr()), d_in.numel(), fmt, bw,
                                      ctypes.c_void_p(d_out.data_ptr()), d_out.numel() * d_out.element_size(),
                                      ctypes.c_void_p(d_result.data_ptr()), _stream_handle(stream)),
           "ms_compress_noalloc")


def to_numpy_u64(t: torch.Tensor) -> np.ndarray:
    """int64 tensor holding uint64 bits -> numpy uint64."""
    return t.detach().cpu().numpy().view(np.uint64)


def batch_config(cfg=None) -> BatchConfig:
    """BatchConfig from a tuple/dict/BatchConfig (None = the library default)."""
    if cfg is None:
        cfg = DEFAULT_BATCH_CONFIG
    if isinstance(cfg, BatchConfig):
        return cfg
    if isinstance(cfg, dict):
        return BatchConfig(**cfg)
    return BatchConfig(*cfg)


class Graph:
    """An instantiated CUDA graph of a batch run (opaque ms_graph*)."""

    def __init__(self, ptr: int):
        self.ptr = ptr

    def launch(self, stream=None):
        _check(load().ms_graph_launch(self.ptr, _stream_handle(stream)), "ms_graph_launch")

    def close(self):
        if self.ptr:
            load().ms_graph_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Fragments sum(y_f[i] for x_f[i] <cmp_f> c1_f (c2_f)) bound to a context's
    columns (ms_batch_*).  Results go to a caller-owned int64 tensor indexed by
    fragment."""

    def __init__(self, ctx: "Ctx", xs, ys, cmps, c1s, c2s=None, stream=None):
        n = len(xs)
        if not (len(ys) == len(cmps) == len(c1s) == n) or (c2s is not None and len(c2s) != n):
            raise ValueError("fragment arrays differ in length")
        self.ctx = ctx
        self.n = n
        self.columns = list(xs) + list(ys)  # keep the handles alive with the batch
        px = (ctypes.c_void_p * n)(*[c.ptr for c in xs])
        py = (ctypes.c_void_p * n)(*[c.ptr for c in ys])
        cmp = np.ascontiguousarray(cmps, dtype=np.int32)
        c1 = np.ascontiguousarray(np.asarray(c1s, dtype=np.uint64))
        c2 = np.ascontiguousarray(np.asarray(c2s if c2s is not None else np.zeros(n), dtype=np.uint64))
        out = ctypes.c_void_p()
        _check(load().ms_batch_create(ctx.h, n, px, py, cmp.ctypes.data_as(ctypes.c_void_p),
                                      c1.ctypes.data_as(ctypes.c_void_p), c2.ctypes.data_as(ctypes.c_void_p),
                                      ctypes.byref(out), _stream_handle(stream)), "ms_batch_create", ctx.h)
        self.ptr = out.value
        if not hasattr(ctx, "_batches"):
            ctx._batches = []
        ctx._batches.append(weakref.ref(self))

    def info(self) -> dict:
        r, c, b = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        _check(load().ms_batch_info(self.ptr, ctypes.byref(r), ctypes.byref(c), ctypes.byref(b)), "ms_batch_info")
        return {"rows": r.value, "chunks": c.value, "bytes": b.value}

    def run(self, sums: torch.Tensor, cfg=None, f0: int = 0, f1: int | None = None, zero: bool = True,
            per_fragment: bool = False, stream=None) -> torch.Tensor:
        f1 = self.n if f1 is None else f1
        assert sums.is_cuda and sums.dtype == torch.int64 and sums.numel() >= self.n
        flags = (BATCH_ZERO if zero else 0) | (BATCH_PER_FRAGMENT if per_fragment else 0)
        c = batch_config(cfg)
        _check(load().ms_batch_run(self.ptr, f0, f1, ctypes.byref(c), flags, _dp(sums), _stream_handle(stream)),
               "ms_batch_run", self.ctx.h)
        return sums

    def graph(self, sums: torch.Tensor, cfg=None, f0: int = 0, f1: int | None = None, zero: bool = True,
              per_fragment: bool = False) -> Graph:
        f1 = self.n if f1 is None else f1
        flags = (BATCH_ZERO if zero else 0) | (BATCH_PER_FRAGMENT if per_fragment else 0)
        c = batch_config(cfg)
        out = ctypes.c_void_p()
        _check(load().ms_batch_graph(self.ptr, f0, f1, ctypes.byref(c), flags, _dp(sums), ctypes.byref(out)),
               "ms_batch_graph", self.ctx.h)
        return Graph(out.value)

    def close(self):
        if self.ptr:
            load().ms_batch_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
