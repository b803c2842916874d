"""Allocator failure injected on the host: the caller's allocation hook refuses a
request, and the library reports MS_ERR_NOMEM, hands back every block it had taken
and leaves the context usable.  No device fault is involved: the hook just returns
NULL."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2004_09350_gb300 import morphstore as ms

pytestmark = pytest.mark.gpu


class Hooks:
    """Allocation hooks backed by torch tensors that refuse every request from the
    `fail_from`-th on (0-based)."""

    def __init__(self, fail_from):
        self.fail_from = fail_from
        self.calls = 0
        self.blocks = {}
        self.unknown_frees = []

        def alloc(size, user):
            i = self.calls
            self.calls += 1
            if i >= self.fail_from:
                return None
            t = torch.empty(int(size), dtype=torch.uint8, device="cuda:0")
            self.blocks[t.data_ptr()] = t
            return t.data_ptr()

        def free(ptr, user):
            if self.blocks.pop(int(ptr), None) is None:
                self.unknown_frees.append(int(ptr))

        self.alloc_cb, self.free_cb = ms._ALLOC_FN(alloc), ms._FREE_FN(free)


def create(h):
    out = ctypes.c_void_p()
    st = ms.load().ms_ctx_create(ctypes.byref(out), 0, 1 << 20, 1 << 12, h.alloc_cb, h.free_cb, None)
    return st, out


@pytest.mark.parametrize("fail_from", [0, 1, 2, 3])
def test_context_creation_reports_nomem_and_returns_every_block(fail_from):
    # creation takes four blocks: arena, control block, column table, work buffer
    h = Hooks(fail_from)
    st, out = create(h)
    assert st == ms.MS_ERR_NOMEM and not out.value
    assert h.calls == 4 if fail_from == 3 else h.calls >= fail_from + 1
    assert h.blocks == {} and h.unknown_frees == []


def test_refused_import_leaves_the_context_usable():
    h = Hooks(4)
    st, ctx = create(h)
    assert st == ms.MS_OK
    L = ms.load()
    data = np.arange(100, dtype=np.uint64) * np.uint64(7)
    col = ctypes.c_void_p()
    assert L.ms_column_import(ctx, ms.UNCOMPR, 0, data.size, ctypes.c_void_p(data.ctypes.data), data.nbytes,
                              ctypes.byref(col), None) == ms.MS_ERR_NOMEM
    assert not col.value
    h.fail_from = 1 << 30
    assert L.ms_column_import(ctx, ms.UNCOMPR, 0, data.size, ctypes.c_void_p(data.ctypes.data), data.nbytes,
                              ctypes.byref(col), None) == ms.MS_OK
    buf = np.zeros(data.nbytes, dtype=np.uint8)
    got = ctypes.c_uint64()
    assert L.ms_column_export(ctx, col, ctypes.c_void_p(buf.ctypes.data), buf.size, ctypes.byref(got), None) == ms.MS_OK
    assert got.value == data.nbytes
    np.testing.assert_array_equal(buf.view(np.uint64), data)
    assert L.ms_get_error(ctx, None) == ms.MS_OK
    assert L.ms_column_free(ctx, col, None) == ms.MS_OK
    assert L.ms_ctx_destroy(ctx) == ms.MS_OK
    assert h.blocks == {} and h.unknown_frees == []
