"""GPU parity of ms_morph (Sec. 3.2, on-the-fly morphing): every ordered pair of
formats, through the C ABI, against the oracle.

A morph from format f1 to f2 must give exactly the bytes the oracle writes when it
compresses the column's values into f2 (the plain definition: the values are
unchanged, only their representation).  Sizes span several 4096-value tiles and a
ragged tail; the value mixes cover unsorted data of skewed widths, sorted keys,
constant blocks and full 64-bit values.
"""
import numpy as np
import pytest

import oracle
from paper_2004_09350_gb300 import morphstore as ms
from paper_2004_09350_gb300 import synth

pytestmark = pytest.mark.gpu

FMTS = [ms.UNCOMPR, ms.STATIC_BP, ms.DYN_BP, ms.DELTA_BP, ms.FOR_BP]


@pytest.fixture(scope="module")
def ctx():
    c = ms.Ctx(0, arena_bytes=1 << 30, max_rows=1 << 20)
    yield c
    c.close()


def _data(kind, n):
    if kind == "skewed":
        return synth.skewed_widths(3, n)
    if kind == "sorted":
        return synth.sorted_gaps(4, n)
    if kind == "flat":
        return np.repeat(synth.splitmix64(5, n // 512 + 1) >> np.uint64(20), 512)[:n].copy()
    return synth.splitmix64(6, n)  # full 64-bit values


def _bw(x):
    return max(1, int(x.max()).bit_length()) if x.size else 1


@pytest.mark.parametrize("src", FMTS)
@pytest.mark.parametrize("dst", FMTS)
@pytest.mark.parametrize("kind,n", [("skewed", 5 * 4096 + 300), ("sorted", 3 * 4096 + 17), ("flat", 4096 + 512),
                                    ("wide", 2 * 4096 + 511), ("skewed", 0), ("sorted", 700)])
def test_morph_every_format_pair(ctx, src, dst, kind, n):
    x = _data(kind, n)
    bw = _bw(x)
    col = ctx.compress(ms.as_device_u64(x, ctx.device), src, bw if src == ms.STATIC_BP else 0)
    out = ctx.morph(col, dst, bw if dst == ms.STATIC_BP else 0)
    ctx.check(what="morph")
    want = oracle.compress(dst, x, bw if dst == ms.STATIC_BP else 0)
    assert ctx.export_bytes(out).tobytes() == want.tobytes()
    np.testing.assert_array_equal(ms.to_numpy_u64(ctx.decompress(out)), x)
    ctx.free(out)
    ctx.free(col)


def test_morph_to_narrow_static_bp_reports_too_wide(ctx):
    x = synth.skewed_widths(7, 3000)
    col = ctx.compress(ms.as_device_u64(x, ctx.device), ms.DYN_BP)
    out = ctx.morph(col, ms.STATIC_BP, _bw(x) - 1)
    assert ctx.get_error() == ms.MS_ERR_VALUE_TOO_WIDE
    ctx.free(out)
    ctx.free(col)
