"""GPU parity of the specialized select on packed codes (ms_select_packed, Sec. 3.2
"Specialized Operators") against oracle.select: every block format and static
BP, every width 1..64, every predicate, with constants that put blocks wholly
inside, wholly outside and across the predicate's range.  The positions are
compared value by value (integer work: bit-exact), and against ms_select."""
import numpy as np
import pytest

import oracle
from paper_2004_09350_gb300 import morphstore as ms
from paper_2004_09350_gb300 import synth

pytestmark = pytest.mark.gpu

N = 3 * 4096 + 777
PACKED = [ms.STATIC_BP, ms.DYN_BP, ms.FOR_BP, ms.DELTA_BP]


@pytest.fixture(scope="module")
def ctx():
    c = ms.Ctx(0, arena_bytes=1 << 30, max_rows=1 << 20)
    yield c
    c.close()


def _column(fmt, b, n=N, seed=11):
    """Values of at most b bits: a mix of random blocks, constant blocks and blocks
    offset by a large reference (FOR), or a sorted column (DELTA)."""
    top = np.uint64((1 << b) - 1) if b < 64 else np.uint64(~np.uint64(0))
    r = synth.splitmix64(seed, n) & top
    if fmt == ms.DELTA_BP:
        step = max(1, (1 << min(b, 40)) // (4 * n) if b < 64 else 1 << 20)
        gaps = (synth.splitmix64(seed + 1, n) % np.uint64(2 * step)).astype(np.uint64)
        x = np.cumsum(gaps, dtype=np.uint64)
        x &= top
        return np.sort(x)
    blk = np.arange(n) // 512
    x = r.copy()
    x[blk % 4 == 1] = r[blk % 4 == 1] & (top >> np.uint64(min(b, 63) // 2))   # narrower blocks
    x[blk % 4 == 2] = r[(blk % 4 == 2).argmax()]                                  # constant blocks
    if fmt == ms.FOR_BP and b < 60:
        x[blk % 4 == 3] = (r[blk % 4 == 3] >> np.uint64(4)) + top - (top >> np.uint64(4))  # high narrow range
    return x


def _predicates(x):
    q = np.quantile(x.astype(np.float64), [0.0, 0.1, 0.5, 0.9, 1.0]) if x.size else [0] * 5
    cs = sorted({int(min(int(v), (1 << 64) - 1)) for v in q} | {0, int(x.max()), int(x.max()) + 1 if int(x.max()) < (1 << 64) - 1 else 0})
    out = []
    for c in cs:
        for cmp in (oracle.EQ, oracle.NE, oracle.LT, oracle.LE, oracle.GT, oracle.GE):
            out.append((cmp, c, 0))
    for lo, hi in ((cs[0], cs[-1]), (cs[1] if len(cs) > 1 else 0, cs[-2] if len(cs) > 1 else 0), (5, 3)):
        out.append((oracle.BETWEEN, lo, hi))
    return out


@pytest.mark.parametrize("fmt", PACKED)
@pytest.mark.parametrize("b", list(range(1, 65)))
def test_select_packed_matches_oracle(ctx, fmt, b):
    x = _column(fmt, b)
    bw = max(1, int(x.max()).bit_length())
    col = ctx.compress(ms.as_device_u64(x, ctx.device), fmt, bw if fmt == ms.STATIC_BP else 0)
    for cmp, c1, c2 in _predicates(x):
        pos = ctx.select_packed(col, cmp, c1, c2, fmt=ms.DELTA_BP)
        got = ms.to_numpy_u64(ctx.decompress(pos))
        ctx.check(what=f"select_packed cmp={cmp} c1={c1} c2={c2}")
        np.testing.assert_array_equal(got, oracle.select(x, cmp, c1, c2), err_msg=f"cmp={cmp} c1={c1} c2={c2}")
        ctx.free(pos)
    ctx.free(col)


@pytest.mark.parametrize("fmt", PACKED)
@pytest.mark.parametrize("n", [0, 1, 511, 512, 513, 4097])
def test_select_packed_edge_lengths(ctx, fmt, n):
    x = synth.sorted_gaps(3, n) if fmt == ms.DELTA_BP else synth.skewed_widths(3, n)
    bw = max(1, int(x.max()).bit_length()) if n else 1
    col = ctx.compress(ms.as_device_u64(x, ctx.device), fmt, bw if fmt == ms.STATIC_BP else 0)
    c = int(np.median(x)) if n else 0
    for cmp in range(7):
        pos = ctx.select_packed(col, cmp, c, c + 7, fmt=ms.DYN_BP)
        ref = ctx.select(col, cmp, c, c + 7, fmt=ms.DYN_BP)
        ctx.check(what="select_packed")
        want = oracle.select(x, cmp, c, c + 7)
        np.testing.assert_array_equal(ms.to_numpy_u64(ctx.decompress(pos)), want)
        assert ctx.export_bytes(pos).tobytes() == ctx.export_bytes(ref).tobytes()
        ctx.free(ref)
        ctx.free(pos)
    ctx.free(col)


def test_select_packed_rejects_uncompressed(ctx):
    col = ctx.compress(ms.as_device_u64(np.arange(100, dtype=np.uint64), ctx.device), ms.UNCOMPR)
    with pytest.raises(ms.MSError) as e:
        ctx.select_packed(col, ms.LT, 5)
    assert e.value.code == ms.MS_ERR_FORMAT
    ctx.free(col)
