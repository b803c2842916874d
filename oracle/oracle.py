"""ctypes wrapper around the plain C oracle (test infrastructure only).

Builds ``liboracle.so`` from ``oracle.c`` with gcc on first use.  Arrays are numpy
``uint64``; compressed columns are numpy ``uint8`` byte arrays in the layout
described at the top of ``oracle.c``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_HDR = os.path.join(_HERE, "oracle.h")
# ORACLE_LIB names a prebuilt oracle library to load instead (a sanitizer build in the tests)
_LIB = os.environ.get("ORACLE_LIB") or os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

UNCOMPR, STATIC_BP, DYN_BP, DELTA_BP, FOR_BP = range(5)
FORMAT_NAMES = ("uncompr", "static_bp", "dyn_bp", "delta_bp", "for_bp")
RLE = 5  # run-length encoding (values, run ends, block directory); not among the five above
FOR_STATIC_BP, DELTA_STATIC_BP = 6, 7  # FOR / DELTA cascaded with static BP (every block at width bw)
EQ, NE, LT, LE, GT, GE, BETWEEN = range(7)
ADD, SUB, MUL = range(3)
OK, BAD_ARG, BAD_FORMAT, TOO_WIDE, OUT_OF_RANGE = range(5)
BLOCK = 512


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"oracle {what} failed with status {code}")
        self.code = code


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, portable; no target-specific flags)."""
    with _lock:
        stale = (not os.path.exists(_LIB) or
                 os.path.getmtime(_LIB) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
        if force or stale:
            tmp = _LIB + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC",
                                   "-o", tmp, _SRC])
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        if not os.environ.get("ORACLE_LIB"):
            build()
        lib = ctypes.CDLL(_LIB)
        u64, i32, p = ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p
        sig = {
            "orc_bitwidth": (i32, [u64]),
            "orc_size": (u64, [i32, i32, p, u64]),
            "orc_compress": (i32, [i32, i32, p, u64, p, u64, p]),
            "orc_decompress": (i32, [i32, i32, u64, p, u64, p]),
            "orc_block_widths": (None, [i32, p, u64, p]),
            "orc_select": (i32, [p, u64, i32, u64, u64, p, p]),
            "orc_project": (i32, [p, u64, p, u64, p]),
            "orc_calc": (i32, [i32, p, p, u64, u64, p]),
            "orc_agg_sum": (u64, [p, u64]),
            "orc_group_sum": (i32, [p, p, u64, u64, p]),
            "orc_semijoin": (i32, [p, u64, p, u64, u64, p, p]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _u64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.uint64))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def bitwidth(x: int) -> int:
    return _load().orc_bitwidth(int(x))


def size(fmt: int, x, bw: int = 0) -> int:
    x = _u64(x)
    return int(_load().orc_size(fmt, bw, _ptr(x), x.size))


def compress(fmt: int, x, bw: int = 0) -> np.ndarray:
    x = _u64(x)
    cap = max(size(fmt, x, bw), 1)
    out = np.zeros(cap, dtype=np.uint8)
    got = ctypes.c_uint64(0)
    rc = _load().orc_compress(fmt, bw, _ptr(x), x.size, _ptr(out), cap, ctypes.byref(got))
    if rc != OK:
        raise OracleError(rc, "compress")
    return out[: got.value]


def decompress(fmt: int, n: int, buf, bw: int = 0) -> np.ndarray:
    buf = np.ascontiguousarray(np.asarray(buf, dtype=np.uint8))
    out = np.zeros(max(n, 1), dtype=np.uint64)
    rc = _load().orc_decompress(fmt, bw, n, _ptr(buf), buf.size, _ptr(out))
    if rc != OK:
        raise OracleError(rc, "decompress")
    return out[:n]


def block_widths(fmt: int, x) -> np.ndarray:
    x = _u64(x)
    out = np.zeros(max(x.size // BLOCK, 1), dtype=np.uint8)
    _load().orc_block_widths(fmt, _ptr(x), x.size, _ptr(out))
    return out[: x.size // BLOCK]


def select(x, cmp: int, c1: int, c2: int = 0) -> np.ndarray:
    x = _u64(x)
    pos = np.zeros(max(x.size, 1), dtype=np.uint64)
    m = ctypes.c_uint64(0)
    rc = _load().orc_select(_ptr(x), x.size, cmp, c1, c2, _ptr(pos), ctypes.byref(m))
    if rc != OK:
        raise OracleError(rc, "select")
    return pos[: m.value].copy()


def project(d, pos) -> np.ndarray:
    d, pos = _u64(d), _u64(pos)
    out = np.zeros(max(pos.size, 1), dtype=np.uint64)
    rc = _load().orc_project(_ptr(d), d.size, _ptr(pos), pos.size, _ptr(out))
    if rc != OK:
        raise OracleError(rc, "project")
    return out[: pos.size]


def calc(op: int, a, b=None, c: int = 0) -> np.ndarray:
    a = _u64(a)
    bb = None if b is None else _u64(b)
    if bb is not None and bb.size != a.size:
        raise OracleError(BAD_ARG, "calc")
    out = np.zeros(max(a.size, 1), dtype=np.uint64)
    rc = _load().orc_calc(op, _ptr(a), None if bb is None else _ptr(bb), c, a.size, _ptr(out))
    if rc != OK:
        raise OracleError(rc, "calc")
    return out[: a.size]


def agg_sum(x) -> int:
    x = _u64(x)
    return int(_load().orc_agg_sum(_ptr(x), x.size))


def group_sum(g, v, n_groups: int) -> np.ndarray:
    g, v = _u64(g), _u64(v)
    if g.size != v.size:
        raise OracleError(BAD_ARG, "group_sum")
    sums = np.zeros(max(n_groups, 1), dtype=np.uint64)
    rc = _load().orc_group_sum(_ptr(g), _ptr(v), g.size, n_groups, _ptr(sums))
    if rc != OK:
        raise OracleError(rc, "group_sum")
    return sums[:n_groups]


def semijoin(probe, keys, key_domain: int) -> np.ndarray:
    probe, keys = _u64(probe), _u64(keys)
    pos = np.zeros(max(probe.size, 1), dtype=np.uint64)
    m = ctypes.c_uint64(0)
    rc = _load().orc_semijoin(_ptr(probe), probe.size, _ptr(keys), keys.size, key_domain,
                              _ptr(pos), ctypes.byref(m))
    if rc != OK:
        raise OracleError(rc, "semijoin")
    return pos[: m.value].copy()


def sizes_all_formats(x) -> dict:
    """Physical size of x under each format (static BP at the column's max width)."""
    x = _u64(x)
    bmax = max(1, bitwidth(int(x.max()))) if x.size else 1
    return {FORMAT_NAMES[f]: size(f, x, bmax if f == STATIC_BP else 0) for f in range(5)}


def best_format_by_size(x) -> str:
    """Exhaustive try-all-formats choice under the footprint objective (Sec. 5.2)."""
    s = sizes_all_formats(x)
    return min(s, key=lambda k: (s[k], FORMAT_NAMES.index(k)))
