"""GPU parity of the RLE format and of FOR / DELTA cascaded with static BP (Sec. 2.1)
through the C ABI, against the oracle.

Encoding (ms_compress, ms_morph from every format) must give exactly the oracle's
bytes: run values, exclusive run ends and the per-block run directory.  Decoding
(ms_decompress, ms_morph to every format) and every operator that reads an RLE
column (select, semi-join probe, project of RLE data and of RLE positions, calc,
agg_sum, group_sum) must give the oracle's results on the plain values.  Sizes span
several 65,536-row claims of the tile stream and a ragged tail; run mixes go from
every value its own run to runs longer than a block.
"""
import numpy as np
import pytest

import oracle
from paper_2004_09350_gb300 import morphstore as ms
from paper_2004_09350_gb300 import synth

pytestmark = pytest.mark.gpu

FMTS = [ms.UNCOMPR, ms.STATIC_BP, ms.DYN_BP, ms.DELTA_BP, ms.FOR_BP]
SIZES = [0, 1, 511, 512, 513, 5 * 4096 + 300, 3 * 65536 + 777]
MEANS = [1, 3, 40, 700, 100_000]


@pytest.fixture(scope="module")
def ctx():
    c = ms.Ctx(0, arena_bytes=1 << 30, max_rows=1 << 20)
    yield c
    c.close()


def _bw(x):
    return max(1, int(x.max()).bit_length()) if x.size else 1


def _col(ctx, x, fmt):
    return ctx.compress(ms.as_device_u64(x, ctx.device), fmt, _bw(x) if fmt == ms.STATIC_BP else 0)


def _values(ctx, col):
    return ms.to_numpy_u64(ctx.decompress(col))


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("mean_run", MEANS)
def test_compress_rle_matches_oracle_bytes(ctx, n, mean_run):
    x = synth.runs(n + mean_run, n, mean_run, distinct=6 if mean_run > 1 else 1 << 40)
    col = _col(ctx, x, ms.RLE)
    ctx.check(what="compress rle")
    assert ctx.export_bytes(col).tobytes() == oracle.compress(oracle.RLE, x).tobytes()
    info = ctx.info(col)
    assert info["n"] == n and info["fmt"] == ms.RLE
    np.testing.assert_array_equal(_values(ctx, col), x)
    ctx.free(col)


@pytest.mark.parametrize("src", FMTS)
@pytest.mark.parametrize("mean_run,n", [(1, 3 * 4096 + 17), (40, 5 * 4096 + 300), (700, 3 * 65536 + 777)])
def test_morph_to_and_from_rle(ctx, src, mean_run, n):
    x = synth.runs(7 * mean_run + src, n, mean_run, distinct=1 << 20)
    bw = _bw(x)
    col = _col(ctx, x, src)
    rle = ctx.morph(col, ms.RLE)
    ctx.check(what="morph to rle")
    assert ctx.export_bytes(rle).tobytes() == oracle.compress(oracle.RLE, x).tobytes()
    back = ctx.morph(rle, src, bw if src == ms.STATIC_BP else 0)
    ctx.check(what="morph from rle")
    assert ctx.export_bytes(back).tobytes() == oracle.compress(src, x, bw if src == ms.STATIC_BP else 0).tobytes()
    ctx.free(back)
    ctx.free(rle)
    ctx.free(col)


def test_import_oracle_bytes_and_reject_bad_sizes(ctx):
    x = synth.runs(11, 4096 + 77, 25)
    buf = oracle.compress(oracle.RLE, x)
    col = ctx.import_bytes(ms.RLE, x.size, buf)
    np.testing.assert_array_equal(_values(ctx, col), x)
    assert ctx.info(col)["n_blocks"] == 1 + int(np.count_nonzero(np.diff(x)))
    ctx.free(col)
    with pytest.raises(ms.MSError) as e:
        ctx.import_bytes(ms.RLE, x.size, buf[:-8])  # not 16 R + 8 ceil(n / 512) bytes
    assert e.value.code == ms.MS_ERR_FORMAT


@pytest.mark.parametrize("mean_run", [1, 40, 700])
@pytest.mark.parametrize("out_fmt", FMTS)
def test_select_on_rle(ctx, mean_run, out_fmt):
    n = 3 * 65536 + 777
    x = synth.runs(21 + mean_run, n, mean_run, distinct=50)
    col = _col(ctx, x, ms.RLE)
    for cmp, c1, c2 in [(ms.LT, 20, 0), (ms.EQ, 7, 0), (ms.BETWEEN, 10, 30), (ms.GE, 49, 0)]:
        out = ctx.select(col, cmp, c1, c2, fmt=out_fmt, bw=max(1, n.bit_length()) if out_fmt == ms.STATIC_BP else 0)
        ctx.check(what="select on rle")
        np.testing.assert_array_equal(_values(ctx, out), oracle.select(x, cmp, c1, c2))
        ctx.free(out)
    ctx.free(col)


@pytest.mark.parametrize("mean_run", [1, 40, 700, 100_000])
def test_agg_sum_of_rle(ctx, mean_run):
    n = 3 * 65536 + 777
    x = synth.runs(31 + mean_run, n, mean_run, distinct=1 << 40)
    col = _col(ctx, x, ms.RLE)
    assert int(ctx.agg_sum(col).item()) & ((1 << 64) - 1) == oracle.agg_sum(x)
    ctx.free(col)


@pytest.mark.parametrize("pos_fmt", FMTS + [ms.RLE])
@pytest.mark.parametrize("mean_run", [1, 40, 100_000])
def test_project_rle_data(ctx, pos_fmt, mean_run):
    """RLE data at sorted positions (a select's output) and at unsorted positions with
    repeats; the positions themselves in every format, RLE included."""
    n = 3 * 65536 + 777
    x = synth.runs(41 + mean_run, n, mean_run, distinct=1 << 30)
    data = _col(ctx, x, ms.RLE)
    sorted_pos = np.sort(synth.uniform(42, 20_000, 0, n))
    unsorted_pos = synth.uniform(43, 20_000, 0, n)
    for pos in (sorted_pos, unsorted_pos):
        pc = _col(ctx, pos, pos_fmt)
        for out_fmt in (ms.UNCOMPR, ms.DYN_BP):
            out = ctx.project(data, pc, fmt=out_fmt)
            ctx.check(what="project rle data")
            np.testing.assert_array_equal(_values(ctx, out), oracle.project(x, pos))
            ctx.free(out)
        ctx.free(pc)
    ctx.free(data)


def test_calc_group_sum_and_semijoin_on_rle(ctx):
    n = 2 * 65536 + 333
    a = synth.runs(51, n, 30, distinct=1 << 20)
    b = synth.uniform(52, n, 0, 1 << 20)
    g = synth.runs(53, n, 200, distinct=105)
    ca, cb, cg = _col(ctx, a, ms.RLE), _col(ctx, b, ms.DYN_BP), _col(ctx, g, ms.RLE)
    out = ctx.calc(ms.MUL, ca, cb, fmt=ms.DYN_BP)
    np.testing.assert_array_equal(_values(ctx, out), oracle.calc(oracle.MUL, a, b))
    ctx.free(out)
    out = ctx.calc(ms.ADD, ca, None, 5, fmt=ms.UNCOMPR)
    np.testing.assert_array_equal(_values(ctx, out), oracle.calc(oracle.ADD, a, None, 5))
    ctx.free(out)
    sums = ms.to_numpy_u64(ctx.group_sum(cg, ca, 105))
    np.testing.assert_array_equal(sums, oracle.group_sum(g, a, 105))
    keys = np.sort(synth.uniform(54, 40, 0, 105))
    ck = _col(ctx, keys, ms.UNCOMPR)
    out = ctx.semijoin(cg, ck, 105, fmt=ms.DELTA_BP)
    ctx.check(what="semijoin rle probe")
    np.testing.assert_array_equal(_values(ctx, out), oracle.semijoin(g, keys, 105))
    ctx.free(out)
    ctx.free(ck)
    ctx.free(cg)
    ctx.free(cb)
    ctx.free(ca)


def test_rle_outputs_and_packed_select_are_refused(ctx):
    x = synth.runs(61, 5000, 10)
    col = _col(ctx, x, ms.RLE)
    for call in (lambda: ctx.select(col, ms.LT, 3, fmt=ms.RLE),
                 lambda: ctx.calc(ms.ADD, col, None, 1, fmt=ms.RLE),
                 lambda: ctx.select_packed(col, ms.LT, 3)):
        with pytest.raises(ms.MSError) as e:
            call()
        assert e.value.code == ms.MS_ERR_FORMAT
    ctx.check(what="refusals leave no device error")
    ctx.free(col)


def test_full_size_rle_sampled():
    """2^27 rows of long runs (the shape of a sorted low-cardinality column): the run
    count and the run-weighted sum against numpy, and 65,536 sampled values (project at
    random positions) against the generating array."""
    n = 1 << 27
    x = synth.runs(71, n, 4000, distinct=1 << 20)
    with ms.Ctx(0, arena_bytes=1 << 31, max_rows=n) as c:
        col = _col(c, x, ms.RLE)
        c.check(what="full-size rle")
        info = c.info(col)
        runs = 1 + int(np.count_nonzero(np.diff(x)))
        assert info["n_blocks"] == runs and info["size_bytes"] == 16 * runs + 8 * (n // 512)
        assert int(c.agg_sum(col).item()) & ((1 << 64) - 1) == int(x.sum(dtype=np.uint64))
        pos = np.sort(synth.uniform(72, 1 << 16, 0, n))
        pc = _col(c, pos, ms.DELTA_BP)
        out = c.project(col, pc, fmt=ms.UNCOMPR)
        np.testing.assert_array_equal(_values(c, out), x[pos.astype(np.int64)])


# ----------------------------------------------- FOR / DELTA cascaded with static BP

CASCADES = [ms.FOR_STATIC_BP, ms.DELTA_STATIC_BP]


def _cascade_data(fmt, n, seed):
    return synth.sorted_gaps(seed, n) if fmt == ms.DELTA_STATIC_BP else synth.table1_column("C3", n, seed)


def _cascade_width(fmt, x):
    base = oracle.DELTA_BP if fmt == ms.DELTA_STATIC_BP else oracle.FOR_BP
    return int(oracle.block_widths(base, x).max()) if x.size >= 512 else 1


@pytest.mark.parametrize("fmt", CASCADES)
@pytest.mark.parametrize("n", [0, 1, 511, 512, 513, 5 * 4096 + 300, 3 * 65536 + 777])
@pytest.mark.parametrize("extra", [0, 5])
def test_compress_static_cascade_matches_oracle_bytes(ctx, fmt, n, extra):
    x = _cascade_data(fmt, n, 81 + n)
    bw = _cascade_width(fmt, x) + extra
    col = ctx.compress(ms.as_device_u64(x, ctx.device), fmt, bw)
    ctx.check(what="compress static cascade")
    assert ctx.export_bytes(col).tobytes() == oracle.compress(fmt, x, bw=bw).tobytes()
    info = ctx.info(col)
    assert info["fmt"] == fmt and info["static_bw"] == bw
    np.testing.assert_array_equal(_values(ctx, col), x)
    ctx.free(col)


@pytest.mark.parametrize("fmt", CASCADES)
def test_static_cascade_too_wide(ctx, fmt):
    x = _cascade_data(fmt, 3000, 83)
    col = ctx.compress(ms.as_device_u64(x, ctx.device), fmt, _cascade_width(fmt, x) - 1)
    assert ctx.get_error() == ms.MS_ERR_VALUE_TOO_WIDE
    ctx.free(col)


@pytest.mark.parametrize("fmt", CASCADES)
@pytest.mark.parametrize("other", FMTS + [ms.RLE])
def test_morph_static_cascade_pairs(ctx, fmt, other):
    n = 5 * 4096 + 300
    x = _cascade_data(fmt, n, 84)
    bw = _cascade_width(fmt, x) + 2
    bwx = _bw(x)
    src = _col(ctx, x, other)
    c = ctx.morph(src, fmt, bw)
    ctx.check(what="morph to cascade")
    assert ctx.export_bytes(c).tobytes() == oracle.compress(fmt, x, bw=bw).tobytes()
    back = ctx.morph(c, other, bwx if other == ms.STATIC_BP else 0)
    ctx.check(what="morph from cascade")
    assert ctx.export_bytes(back).tobytes() == oracle.compress(other, x, bwx if other == ms.STATIC_BP else 0).tobytes()
    ctx.free(back)
    ctx.free(c)
    ctx.free(src)


@pytest.mark.parametrize("fmt", CASCADES)
def test_operators_read_static_cascades(ctx, fmt):
    """select (general and on the packed codes), agg_sum, project (as data and as the
    position list) and calc on the cascades, against the oracle."""
    n = 3 * 65536 + 777
    x = _cascade_data(fmt, n, 85)
    bw = _cascade_width(fmt, x) + 1
    col = ctx.compress(ms.as_device_u64(x, ctx.device), fmt, bw)
    c = synth.value_at_rank(x, 0.3)
    for sel in (ctx.select, ctx.select_packed):
        out = sel(col, ms.LT, c, fmt=ms.DELTA_BP)
        np.testing.assert_array_equal(_values(ctx, out), oracle.select(x, oracle.LT, c))
        ctx.free(out)
    assert int(ctx.agg_sum(col).item()) & ((1 << 64) - 1) == oracle.agg_sum(x)
    pos = np.sort(synth.uniform(86, 30_000, 0, n))
    pc = ctx.compress(ms.as_device_u64(pos, ctx.device), ms.DELTA_STATIC_BP, _cascade_width(ms.DELTA_STATIC_BP, pos))
    out = ctx.project(col, pc, fmt=fmt, bw=_bw(x))
    np.testing.assert_array_equal(_values(ctx, out), oracle.project(x, pos))
    ctx.free(out)
    out = ctx.calc(ms.ADD, col, None, 7, fmt=fmt, bw=bw)
    np.testing.assert_array_equal(_values(ctx, out), oracle.calc(oracle.ADD, x, None, 7))
    ctx.free(out)
    ctx.free(pc)
    ctx.free(col)
