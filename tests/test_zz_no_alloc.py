"""ms_compress_noalloc against ms_compress, through the C ABI.

ms_compress_noalloc serves callers that cannot allocate device memory: for
example, a memory manager compressing a buffer while it serves an allocation
request, or a host whose device memory all belongs to its own pool.  Its scratch
is a fixed device array inside the library, shared by every call.  These tests
check that two calls in a row produce exactly the bytes the allocating entry
point produces (integer codec: bit-exact is the bar used by every parity test).
This file is collected last so that a stop-at-first-failure run has already run
every other test.
"""
import numpy as np
import pytest
import torch

from paper_2004_09350_gb300 import morphstore as ms
from paper_2004_09350_gb300 import synth

pytestmark = pytest.mark.gpu


def _reference_bytes(ctx, x, fmt, bw):
    col = ctx.compress(ms.as_device_u64(x, ctx.device), fmt, bw)
    ctx.check(what="ms_compress")
    out = ctx.export_bytes(col)
    ctx.free(col)
    return out


@pytest.mark.parametrize("fmt", [ms.DYN_BP, ms.DELTA_BP, ms.FOR_BP, ms.STATIC_BP, ms.UNCOMPR])
def test_noalloc_matches_allocating_entry_point_twice(fmt):
    with ms.Ctx(0, arena_bytes=256 << 20, max_rows=1 << 20) as ctx:
        dev = ctx.device
        for call, (n, seed) in enumerate([(9 * 4096 + 700, 1), (3 * 4096 + 5, 2)]):
            x = synth.skewed_widths(seed, n) if fmt != ms.DELTA_BP else synth.sorted_gaps(seed, n)
            bw = max(1, int(x.max()).bit_length()) if fmt == ms.STATIC_BP else 0
            want = _reference_bytes(ctx, x, fmt, bw)
            d_in = ms.as_device_u64(x, dev)
            d_out = torch.full((want.size + 4096,), 0xA5, dtype=torch.uint8, device=dev)
            d_res = torch.zeros(2, dtype=torch.int64, device=dev)
            ms.compress_noalloc(d_in, fmt, d_out, d_res, bw=bw)
            torch.cuda.synchronize()
            size, status = (int(v) for v in d_res.cpu().tolist())
            assert status == ms.MS_OK, f"call {call}: device status {status}"
            assert size == want.size, f"call {call}"
            got = d_out[:size].cpu().numpy()
            assert got.tobytes() == want.tobytes(), f"call {call}: bytes differ"


def test_noalloc_reports_small_buffer_and_rejects_oversize():
    x = synth.skewed_widths(3, 5000)
    dev = torch.device("cuda", 0)
    d_in = ms.as_device_u64(x, dev)
    d_out = torch.empty(64, dtype=torch.uint8, device=dev)
    d_res = torch.zeros(2, dtype=torch.int64, device=dev)
    ms.compress_noalloc(d_in, ms.DYN_BP, d_out, d_res)
    torch.cuda.synchronize()
    assert int(d_res[1]) == ms.MS_ERR_NOMEM
    big = torch.empty(ms.NOALLOC_MAX_ROWS + 1, dtype=torch.int64, device=dev)
    with pytest.raises(ms.MSError) as e:
        ms.compress_noalloc(big, ms.DYN_BP, d_out, d_res)
    assert e.value.code == ms.MS_ERR_INVALID_ARG
