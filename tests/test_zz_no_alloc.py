"""ms_compress_noalloc through the C ABI, against the oracle and against ms_compress.

ms_compress_noalloc serves callers that cannot allocate device memory: for
example, a memory manager compressing a buffer while it serves an allocation
request (it must not re-enter its own allocator), or a host whose device memory
all belongs to its own pool.  Its scratch is a fixed device array inside the
library, shared by every call and kept between calls.  These tests check that
two calls in a row produce exactly the oracle's bytes (integer codec: bit-exact
is the bar of every parity test here), that the largest accepted column matches
the allocating entry point byte for byte and decodes back to its input in the
oracle, and the empty and error cases.  The file is collected last, so a run
that stops at its first failure has already run every other test.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2004_09350_gb300 import morphstore as ms
from paper_2004_09350_gb300 import synth

pytestmark = pytest.mark.gpu
FORMATS = [ms.DYN_BP, ms.DELTA_BP, ms.FOR_BP, ms.STATIC_BP, ms.UNCOMPR]


def _column(fmt, n, seed):
    x = synth.sorted_gaps(seed, n) if fmt == ms.DELTA_BP else synth.skewed_widths(seed, n)
    bw = max(1, int(x.max()).bit_length()) if fmt == ms.STATIC_BP and n else 0
    return x, bw


def _noalloc(x, fmt, bw, cap_bytes):
    dev = torch.device("cuda", 0)
    d_in = ms.as_device_u64(x, dev)
    d_out = torch.full((cap_bytes,), 0xA5, dtype=torch.uint8, device=dev)
    d_res = torch.zeros(2, dtype=torch.int64, device=dev)
    ms.compress_noalloc(d_in, fmt, d_out, d_res, bw=bw)
    torch.cuda.synchronize()
    size, status = (int(v) for v in d_res.cpu().tolist())
    return size, status, d_out


@pytest.mark.parametrize("fmt", FORMATS)
def test_noalloc_matches_oracle_bytes_twice(fmt):
    # two calls in a row share the scratch array: each must start from a clean state
    for call, (n, seed) in enumerate([(9 * 4096 + 700, 1), (3 * 4096 + 5, 2)]):
        x, bw = _column(fmt, n, seed)
        want = oracle.compress(fmt, x, bw)
        size, status, d_out = _noalloc(x, fmt, bw, want.size + 4096)
        assert status == ms.MS_OK, f"call {call}: device status {status}"
        assert size == want.size, f"call {call}"
        assert d_out[:size].cpu().numpy().tobytes() == want.tobytes(), f"call {call}: bytes differ"


@pytest.mark.parametrize("fmt", FORMATS)
def test_noalloc_at_the_row_limit(fmt):
    # n = MS_NOALLOC_MAX_ROWS uses every look-back status word (4097 tiles of 4096
    # values, so CTAs run several tiles and look-backs walk far); n - 3 adds a ragged
    # remainder.  Bytes equal ms_compress's, and the oracle decodes them to the input.
    with ms.Ctx(0, arena_bytes=(1 << 30) + (256 << 20), max_rows=ms.NOALLOC_MAX_ROWS) as ctx:
        for n in (ms.NOALLOC_MAX_ROWS, ms.NOALLOC_MAX_ROWS - 3):
            x, bw = _column(fmt, n, 7)
            col = ctx.compress(ms.as_device_u64(x, ctx.device), fmt, bw)
            ctx.check(what="ms_compress")
            want = ctx.export_bytes(col)
            ctx.free(col)
            size, status, d_out = _noalloc(x, fmt, bw, want.size + 256)
            assert status == ms.MS_OK and size == want.size, (n, status, size, want.size)
            got = d_out[:size].cpu().numpy()
            assert got.tobytes() == want.tobytes(), f"n={n}: bytes differ from ms_compress"
            np.testing.assert_array_equal(oracle.decompress(fmt, n, got, bw), x)


def test_noalloc_empty_column():
    dev = torch.device("cuda", 0)
    d_out = torch.full((256,), 0xA5, dtype=torch.uint8, device=dev)
    d_res = torch.full((2,), -1, dtype=torch.int64, device=dev)
    for fmt in FORMATS:
        ms.compress_noalloc(torch.empty(0, dtype=torch.int64, device=dev), fmt, d_out, d_res,
                            bw=5 if fmt == ms.STATIC_BP else 0)
        torch.cuda.synchronize()
        assert d_res.cpu().tolist() == [0, ms.MS_OK], fmt


def test_noalloc_reports_errors():
    dev = torch.device("cuda", 0)
    x = synth.skewed_widths(3, 5000)
    d_in = ms.as_device_u64(x, dev)
    d_out = torch.empty(64, dtype=torch.uint8, device=dev)
    d_res = torch.zeros(2, dtype=torch.int64, device=dev)
    ms.compress_noalloc(d_in, ms.DYN_BP, d_out, d_res)  # output buffer too small
    torch.cuda.synchronize()
    assert int(d_res[1]) == ms.MS_ERR_NOMEM
    # static BP narrower than the widest value
    big = torch.empty(1 << 16, dtype=torch.uint8, device=dev)
    ms.compress_noalloc(d_in, ms.STATIC_BP, big, d_res, bw=int(x.max()).bit_length() - 1)
    torch.cuda.synchronize()
    assert int(d_res[1]) == ms.MS_ERR_VALUE_TOO_WIDE
    with pytest.raises(ms.MSError) as e:
        ms.compress_noalloc(torch.empty(ms.NOALLOC_MAX_ROWS + 1, dtype=torch.int64, device=dev), ms.DYN_BP,
                            d_out, d_res)
    assert e.value.code == ms.MS_ERR_INVALID_ARG
    # a later good call is unaffected by the errors before it
    want = oracle.compress(ms.DYN_BP, x)
    size, status, d_out = _noalloc(x, ms.DYN_BP, 0, want.size + 64)
    assert status == ms.MS_OK and d_out[:size].cpu().numpy().tobytes() == want.tobytes()
