"""GPU parity: every operator through the C ABI against the CPU oracle.

Integer work, so the bar is bit-exact: decompressed values, compressed bytes (both
sides implement the same written layout) and aggregates.  Sizes span several
4096-value tiles plus ragged tails; every input/output format pair is covered.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2004_09350_gb300 import morphstore as ms
from paper_2004_09350_gb300 import synth

pytestmark = pytest.mark.gpu

FMTS = [ms.UNCOMPR, ms.STATIC_BP, ms.DYN_BP, ms.DELTA_BP, ms.FOR_BP]


@pytest.fixture(scope="module")
def ctx():
    c = ms.Ctx(0, arena_bytes=3 << 30, max_rows=1 << 22)
    yield c
    c.close()


def static_bw(x):
    return max(1, int(x.max()).bit_length()) if x.size else 1


def gpu_col(ctx, x, fmt, bw=None):
    bw = static_bw(x) if bw is None else bw
    d = ms.as_device_u64(x, ctx.device)
    col = ctx.compress(d, fmt, bw if fmt == ms.STATIC_BP else 0)
    return col, (bw if fmt == ms.STATIC_BP else 0)


def values(ctx, col):
    return ms.to_numpy_u64(ctx.decompress(col))


def assert_column(ctx, col, want, fmt, bw=0):
    ctx.check(what="device error")
    got = values(ctx, col)
    np.testing.assert_array_equal(got, want)
    ref = oracle.compress(fmt, want, bw=bw)
    assert ctx.export_bytes(col).tobytes() == ref.tobytes()


def edge_column(n, b, seed=1):
    if b == 0:
        return np.zeros(n, dtype=np.uint64)
    x = synth.splitmix64(seed, n) >> np.uint64(64 - b)
    if n:
        x[n // 2] |= np.uint64(1) << np.uint64(b - 1)
    return x


NS = [0, 1, 15, 511, 512, 513, 4096, 4097, 3 * 4096 + 777]


# ------------------------------------------------------------------- codecs

@pytest.mark.parametrize("fmt", FMTS)
@pytest.mark.parametrize("n", NS)
@pytest.mark.parametrize("b", [0, 1, 7, 31, 32, 33, 63, 64])
def test_compress_matches_oracle_bytes(ctx, fmt, n, b):
    x = edge_column(n, b, seed=n + b)
    col, bw = gpu_col(ctx, x, fmt)
    assert_column(ctx, col, x, fmt, bw)
    ctx.free(col)


@pytest.mark.parametrize("fmt", FMTS)
@pytest.mark.parametrize("kind", ["skewed", "sorted", "C2", "C3", "C4"])
def test_compress_workload_shapes(ctx, fmt, kind):
    n = 5 * 4096 + 333
    x = {"skewed": lambda: synth.skewed_widths(3, n), "sorted": lambda: synth.sorted_gaps(4, n),
         "C2": lambda: synth.table1_column("C2", n), "C3": lambda: synth.table1_column("C3", n),
         "C4": lambda: synth.table1_column("C4", n)}[kind]()
    col, bw = gpu_col(ctx, x, fmt)
    assert_column(ctx, col, x, fmt, bw)
    info = ctx.info(col)
    assert info["n"] == n and info["size_bytes"] == oracle.size(fmt, x, bw)
    ctx.free(col)


@pytest.mark.parametrize("fmt", FMTS)
@pytest.mark.parametrize("n", [0, 700, 4096 * 2 + 5])
def test_decode_of_oracle_bytes(ctx, fmt, n):
    x = synth.skewed_widths(n + 11, n)
    bw = static_bw(x)
    buf = oracle.compress(fmt, x, bw=bw)
    col = ctx.import_bytes(fmt, n, buf, bw=bw)
    ctx.check()
    np.testing.assert_array_equal(values(ctx, col), x)
    ctx.free(col)


# ------------------------------------------------------------------ select

@pytest.mark.parametrize("in_fmt", FMTS)
@pytest.mark.parametrize("out_fmt", FMTS)
def test_select_every_format_pair(ctx, in_fmt, out_fmt):
    n = 6 * 4096 + 321
    x = synth.skewed_widths(7, n, widths=(3, 8, 16))
    col, _ = gpu_col(ctx, x, in_fmt)
    for sel in (0.001, 0.1, 0.9):
        c = synth.value_at_rank(x, sel)
        want = oracle.select(x, oracle.LT, c)
        bw = static_bw(np.array([n], dtype=np.uint64)) if out_fmt == ms.STATIC_BP else 0
        pos = ctx.select(col, ms.LT, c, fmt=out_fmt, bw=bw)
        assert_column(ctx, pos, want, out_fmt, bw)
        ctx.free(pos)
    ctx.free(col)


@pytest.mark.parametrize("cmp", [ms.EQ, ms.NE, ms.LE, ms.GT, ms.GE, ms.BETWEEN])
def test_select_predicates(ctx, cmp):
    n = 3 * 4096 + 99
    x = synth.uniform(3, n, 0, 50)
    col, _ = gpu_col(ctx, x, ms.DYN_BP)
    pos = ctx.select(col, cmp, 17, 31, fmt=ms.DELTA_BP)
    assert_column(ctx, pos, oracle.select(x, cmp, 17, 31), ms.DELTA_BP)
    ctx.free(pos)
    ctx.free(col)


@pytest.mark.parametrize("out_fmt", FMTS)
def test_select_sparse_output_blocks(ctx, out_fmt):
    """Selectivities below 1/64: an output block of 512 positions gathers from more
    than 64 input chunks (several 32-chunk spans per block, the last span full)."""
    n = 400 * 512 + 77
    x = synth.uniform(13, n, 0, 1 << 30)
    col, _ = gpu_col(ctx, x, ms.DYN_BP)
    for sel in (0.0005, 0.002, 0.01, 0.015, 0.03):
        c = synth.value_at_rank(x, sel)
        want = oracle.select(x, oracle.LT, c)
        bw = static_bw(np.array([n], dtype=np.uint64)) if out_fmt == ms.STATIC_BP else 0
        pos = ctx.select(col, ms.LT, c, fmt=out_fmt, bw=bw)
        assert_column(ctx, pos, want, out_fmt, bw)
        ctx.free(pos)
    ctx.free(col)


NARROW_CASES = [(ms.EQ, 5, 0), (ms.EQ, 1 << 33, 0), (ms.NE, 7, 0), (ms.NE, 1 << 40, 0), (ms.LT, 0, 0),
                (ms.LT, 1 << 40, 0), (ms.LT, 1 << 19, 0), (ms.LE, (1 << 32) - 1, 0), (ms.GT, 2**64 - 1, 0),
                (ms.GT, 1 << 32, 0), (ms.GT, 1000, 0), (ms.GE, 0, 0), (ms.GE, (1 << 32) - 5, 0),
                (ms.BETWEEN, 9, 3), (ms.BETWEEN, 1 << 31, 1 << 33), (ms.BETWEEN, 1 << 33, 1 << 34),
                (ms.BETWEEN, 100, 2**64 - 1), (ms.BETWEEN, 0, 2**64 - 1), (ms.BETWEEN, 1 << 10, 1 << 19)]


@pytest.mark.parametrize("fmt", [ms.DYN_BP, ms.STATIC_BP, ms.FOR_BP])
@pytest.mark.parametrize("case", NARROW_CASES, ids=lambda c: "%d-%d-%d" % c)
def test_select_narrow_predicates(ctx, fmt, case):
    """Blocks of at most 32 bits take the 32-bit form of the range test; constants
    at and beyond 2^32, empty and full ranges, and negations must agree with the
    64-bit definition."""
    cmp, c1, c2 = case
    n = 3 * 4096 + 77
    x = synth.skewed_widths(51, n, widths=(1, 12, 20, 32))
    x[::997] = np.uint64((1 << 32) - 1)
    x[5] = np.uint64((1 << 32) - 5)
    col, _ = gpu_col(ctx, x, fmt)
    pos = ctx.select(col, cmp, c1, c2, fmt=ms.DELTA_BP)
    assert_column(ctx, pos, oracle.select(x, cmp, c1, c2), ms.DELTA_BP)
    ctx.free(pos)
    ctx.free(col)


def test_select_none_and_all(ctx):
    x = synth.uniform(5, 4096 * 4 + 17, 10, 20)
    col, _ = gpu_col(ctx, x, ms.FOR_BP)
    for c, want_n in ((10, 0), (20, x.size)):
        pos = ctx.select(col, ms.LT, c, fmt=ms.DELTA_BP)
        assert ctx.info(pos)["n"] == want_n
        assert_column(ctx, pos, oracle.select(x, oracle.LT, c), ms.DELTA_BP)
        ctx.free(pos)
    ctx.free(col)


# ----------------------------------------------------------------- project

@pytest.mark.parametrize("data_fmt", FMTS)
@pytest.mark.parametrize("out_fmt", FMTS)
def test_project_every_format_pair(ctx, data_fmt, out_fmt):
    n = 5 * 4096 + 123
    d = synth.sorted_gaps(9, n) if data_fmt == ms.DELTA_BP else synth.skewed_widths(9, n)
    dcol, _ = gpu_col(ctx, d, data_fmt)
    pos = np.sort(synth.uniform(10, 3000, 0, n))
    pcol, _ = gpu_col(ctx, pos, ms.DELTA_BP)
    want = oracle.project(d, pos)
    bw = static_bw(want)
    out = ctx.project(dcol, pcol, fmt=out_fmt, bw=bw)
    assert_column(ctx, out, want, out_fmt, bw if out_fmt == ms.STATIC_BP else 0)
    ctx.free(out)
    ctx.free(pcol)
    ctx.free(dcol)


@pytest.mark.parametrize("data_fmt", [ms.STATIC_BP, ms.DYN_BP, ms.FOR_BP])
@pytest.mark.parametrize("step", [1, 3, 20, 70, 200, 2000])
def test_project_sorted_spans(ctx, data_fmt, step):
    """Sorted positions every `step` rows (plus a jitter): an output chunk spans from
    one data block to hundreds of them, so its blocks are staged in one piece, in
    several pieces of wide (40-bit) blocks, or read at random past the span limit;
    positions also reach the uncompressed remainder / static tail."""
    n = 300 * 512 + 301
    d = synth.skewed_widths(41, n, widths=(1, 17, 40, 64)) if data_fmt != ms.STATIC_BP else synth.uniform(41, n, 0, 1 << 40)
    dcol, bw = gpu_col(ctx, d, data_fmt)
    base = np.arange(0, n, step, dtype=np.uint64)
    jit = synth.uniform(42, base.size, 0, max(step // 2, 1))
    pos = np.minimum(base + jit, np.uint64(n - 1))
    pos = np.concatenate([pos, np.arange(n - 40, n, dtype=np.uint64)])
    pos.sort()
    pcol, _ = gpu_col(ctx, pos, ms.DELTA_BP)
    want = oracle.project(d, pos)
    out = ctx.project(dcol, pcol, fmt=ms.DYN_BP)
    assert_column(ctx, out, want, ms.DYN_BP)
    ctx.free(out)
    ctx.free(pcol)
    ctx.free(dcol)


@pytest.mark.parametrize("bw", [1, 5, 17, 23, 32, 33, 34, 64])
def test_project_static_data_at_random(ctx, bw):
    """Static-BP data read in place at sparse sorted and at unsorted positions, at
    widths on both sides of the 33-bit limit of the three-halfword read, with
    positions in the horizontal tail."""
    n = 120 * 512 + 333
    d = edge_column(n, bw, seed=bw)
    dcol, _ = gpu_col(ctx, d, ms.STATIC_BP, bw=bw)
    sparse = np.sort(synth.uniform(57, 1500, 0, n))
    unsorted = synth.uniform(58, 3000, 0, n)
    tail = np.arange(n - 333, n, 7, dtype=np.uint64)
    for pos, pfmt in ((np.concatenate([sparse, tail]), ms.DELTA_BP), (np.concatenate([unsorted, tail]), ms.DYN_BP)):
        pos_s = np.sort(pos) if pfmt == ms.DELTA_BP else pos
        pcol, _ = gpu_col(ctx, pos_s, pfmt)
        out = ctx.project(dcol, pcol, fmt=ms.UNCOMPR)
        assert_column(ctx, out, oracle.project(d, pos_s), ms.UNCOMPR)
        ctx.free(out)
        ctx.free(pcol)
    ctx.free(dcol)


@pytest.mark.parametrize("kind", ["gaps", "random", "flat", "widths"])
@pytest.mark.parametrize("step", [0, 1, 3, 70, 2000])
def test_project_delta_data_sorted_positions(ctx, kind, step):
    """DELTA data read at sorted positions (repeats allowed) block by block: narrow
    blocks (32-bit prefix sums), blocks whose differences wrap modulo 2^64 (64-bit
    sums), blocks of width 0 (answered by their reference), the 22..24-bit switch,
    spans from one block to hundreds, and positions in the raw remainder."""
    n = 200 * 512 + 77
    if kind == "gaps":
        d = synth.sorted_gaps(51, n)
    elif kind == "random":
        d = synth.splitmix64(52, n)
    elif kind == "flat":
        d = np.repeat(synth.uniform(53, n // 700 + 1, 0, 1 << 40), 700)[:n]
    else:
        d = delta_width_column([22, 23, 24, 0, 1, 40, 64] * 28, tail=77)
        n = d.size
    dcol, _ = gpu_col(ctx, d, ms.DELTA_BP)
    if step == 0:  # sorted random positions with repeats
        pos = np.sort(synth.uniform(54, 20_000, 0, n))
    else:
        pos = np.arange(step // 2, n, step, dtype=np.uint64)
    pos = np.concatenate([pos, np.arange(n - 30, n, dtype=np.uint64)])
    pos.sort()
    pcol, _ = gpu_col(ctx, pos, ms.DELTA_BP)
    want = oracle.project(d, pos)
    for out_fmt in (ms.UNCOMPR, ms.DELTA_BP):
        out = ctx.project(dcol, pcol, fmt=out_fmt)
        assert_column(ctx, out, want, out_fmt)
        ctx.free(out)
    ctx.free(pcol)
    ctx.free(dcol)


@pytest.mark.parametrize("data_fmt", FMTS)
@pytest.mark.parametrize("pos_fmt", FMTS)
def test_project_position_formats_and_unsorted(ctx, data_fmt, pos_fmt):
    n = 3 * 4096 + 1000
    d = synth.splitmix64(21, n) >> np.uint64(20)
    dcol, _ = gpu_col(ctx, d, data_fmt)
    pos = synth.uniform(22, 5000, 0, n)  # unsorted, with repeats
    pcol, _ = gpu_col(ctx, pos, pos_fmt)
    out = ctx.project(dcol, pcol, fmt=ms.UNCOMPR)
    assert_column(ctx, out, oracle.project(d, pos), ms.UNCOMPR)
    ctx.free(out)
    ctx.free(pcol)
    ctx.free(dcol)


def delta_width_column(widths, tail=100, seed=5):
    """Blocks of in-block differences at the given widths: even blocks take every
    difference at its maximum 2^b - 1 (512 of them sum to just below 2^32 at b = 23),
    odd ones random differences below 2^b with one at the maximum; block starts sit
    near 2^64 so that the running values wrap."""
    parts, v = [], np.uint64(2**64 - 5)
    for i, b in enumerate(widths):
        top = np.uint64((1 << b) - 1)
        r = np.full(512, top, dtype=np.uint64) if i % 2 == 0 else synth.splitmix64(seed + i, 512) & top
        r[0] = 0
        r[1] = top
        with np.errstate(over="ignore"):
            blk = v + np.cumsum(r, dtype=np.uint64)
        parts.append(blk)
        v = synth.splitmix64(seed + 100 + i, 1)[0] | np.uint64(1 << 63)
    parts.append(synth.splitmix64(seed + 999, tail))
    return np.concatenate(parts)


def test_delta_prefix_sums_at_the_32_bit_boundary(ctx):
    """DELTA blocks of width <= 23 take 32-bit prefix sums, wider ones 64-bit: both
    sides of that switch, at their largest sums, through every DELTA decoder (chunk
    stream, CTA tile stream, project's block decode)."""
    widths = [22, 23, 23, 24, 24, 31, 32, 33, 1, 0, 23, 63, 64, 23]
    x = delta_width_column(widths)
    ref = oracle.compress(ms.DELTA_BP, x)
    hdr = ref.view(np.uint64)[: 2 * len(widths)].reshape(-1, 2)
    assert [int(w) & 255 for w in hdr[:, 0]] == widths
    col, _ = gpu_col(ctx, x, ms.DELTA_BP)
    assert_column(ctx, col, x, ms.DELTA_BP)
    assert int(ms.to_numpy_u64(ctx.agg_sum(col))[0]) == oracle.agg_sum(x)
    ctx.check()
    n = x.size
    for pos in (np.arange(n, dtype=np.uint64), np.arange(3, n, 7, dtype=np.uint64),
                np.sort(synth.uniform(6, 900, 0, n))):
        pcol, _ = gpu_col(ctx, pos, ms.DELTA_BP)
        for out_fmt in (ms.UNCOMPR, ms.DELTA_BP):
            out = ctx.project(col, pcol, fmt=out_fmt)
            assert_column(ctx, out, oracle.project(x, pos), out_fmt)
            ctx.free(out)
        ctx.free(pcol)
    out = ctx.calc(ms.ADD, col, col, fmt=ms.DELTA_BP)
    assert_column(ctx, out, oracle.calc(ms.ADD, x, x), ms.DELTA_BP)
    ctx.free(out)
    ctx.free(col)


# -------------------------------------------------------------------- calc

@pytest.mark.parametrize("fa,fb", [(f, f) for f in FMTS] + [(ms.DYN_BP, ms.DELTA_BP), (ms.UNCOMPR, ms.FOR_BP),
                                                           (ms.STATIC_BP, ms.DYN_BP)])
@pytest.mark.parametrize("op", [ms.ADD, ms.SUB, ms.MUL])
def test_calc_pairs(ctx, fa, fb, op):
    n = 4 * 4096 + 55
    a = synth.skewed_widths(31, n)
    b = synth.sorted_gaps(32, n)
    ca, _ = gpu_col(ctx, a, fa)
    cb, _ = gpu_col(ctx, b, fb)
    want = oracle.calc(op, a, b)
    for out_fmt in (ms.UNCOMPR, ms.DYN_BP, ms.FOR_BP):
        out = ctx.calc(op, ca, cb, fmt=out_fmt)
        assert_column(ctx, out, want, out_fmt)
        ctx.free(out)
    out = ctx.calc(op, ca, None, c=12345, fmt=ms.DELTA_BP)
    assert_column(ctx, out, oracle.calc(op, a, c=12345), ms.DELTA_BP)
    ctx.free(out)
    ctx.free(cb)
    ctx.free(ca)


# --------------------------------------------------------------- aggregates

@pytest.mark.parametrize("fmt", FMTS)
@pytest.mark.parametrize("n", [0, 1, 513, 7 * 4096 + 3])
def test_agg_sum(ctx, fmt, n):
    x = synth.table1_column("C3", n) if fmt != ms.STATIC_BP else synth.skewed_widths(4, n)
    col, _ = gpu_col(ctx, x, fmt)
    got = int(ms.to_numpy_u64(ctx.agg_sum(col))[0])
    ctx.check()
    assert got == oracle.agg_sum(x)
    ctx.free(col)


@pytest.mark.parametrize("fg,fv", [(ms.UNCOMPR, ms.UNCOMPR), (ms.STATIC_BP, ms.DYN_BP), (ms.DYN_BP, ms.FOR_BP),
                                   (ms.FOR_BP, ms.DELTA_BP)])
@pytest.mark.parametrize("G", [1, 105, 5000])
def test_group_sum(ctx, fg, fv, G):
    n = 5 * 4096 + 77
    g = synth.uniform(41, n, 0, G)
    v = synth.splitmix64(42, n)
    cg, _ = gpu_col(ctx, g, fg)
    cv, _ = gpu_col(ctx, v, fv)
    got = ms.to_numpy_u64(ctx.group_sum(cg, cv, G))
    ctx.check()
    np.testing.assert_array_equal(got, oracle.group_sum(g, v, G))
    ctx.free(cv)
    ctx.free(cg)


@pytest.mark.parametrize("probe_fmt", FMTS)
@pytest.mark.parametrize("out_fmt", [ms.UNCOMPR, ms.DELTA_BP, ms.DYN_BP])
def test_semijoin(ctx, probe_fmt, out_fmt):
    n, dom = 6 * 4096 + 999, 30_000
    probe = synth.uniform(51, n, 0, dom)
    keys = np.sort(synth.uniform(52, 4000, 0, dom))
    cp, _ = gpu_col(ctx, probe, probe_fmt)
    ck, _ = gpu_col(ctx, keys, ms.DELTA_BP)
    out = ctx.semijoin(cp, ck, dom, fmt=out_fmt)
    assert_column(ctx, out, oracle.semijoin(probe, keys, dom), out_fmt)
    ctx.free(out)
    ctx.free(ck)
    ctx.free(cp)


@pytest.mark.parametrize("dom", [1_500_000, 3_000_000, 40_000_000])
def test_semijoin_large_key_domains(ctx, dom):
    """Key bitmaps that fit one CTA's shared memory (1.5e6 keys) and larger ones
    probed through L1 and L2 (3e6 keys, 375 KB; 4e7 keys, 5 MB); probe values span
    the whole domain, with some at or beyond its end."""
    n = 9 * 4096 + 313
    probe = synth.uniform(55, n, 0, dom)
    probe[:50] = np.uint64(dom - 1)
    probe[50:60] = np.uint64(dom) + np.arange(10, dtype=np.uint64)
    keys = np.sort(synth.uniform(56, 40_000, 0, dom))
    keys[-1] = dom - 1
    for probe_fmt in (ms.DYN_BP, ms.UNCOMPR):
        cp, _ = gpu_col(ctx, probe, probe_fmt)
        ck, _ = gpu_col(ctx, keys, ms.DELTA_BP)
        out = ctx.semijoin(cp, ck, dom, fmt=ms.DELTA_BP)
        assert_column(ctx, out, oracle.semijoin(probe, keys, dom), ms.DELTA_BP)
        ctx.free(out)
        ctx.free(ck)
        ctx.free(cp)


# ------------------------------------------------------------------ plans

def test_tiny_fragment_plan_bit_exact(ctx):
    """Two 2^20-row columns: A static BP 12 bits, B dynamic BP; select A < 410 ->
    DELTA+BP positions -> project B -> dynamic BP -> sum; and all-uncompressed."""
    a, b = synth.tiny_fragment()
    want_pos = oracle.select(a, oracle.LT, 410)
    want_y = oracle.project(b, want_pos)
    want_sum = oracle.agg_sum(want_y)
    assert abs(want_pos.size - 104_960) < 6 * 307  # Binomial(2^20, 410/4096)
    for fa, fb, fp, fy in ((ms.STATIC_BP, ms.DYN_BP, ms.DELTA_BP, ms.DYN_BP),
                           (ms.UNCOMPR, ms.UNCOMPR, ms.UNCOMPR, ms.UNCOMPR)):
        ca, _ = gpu_col(ctx, a, fa, bw=12)
        cb, _ = gpu_col(ctx, b, fb)
        pos = ctx.select(ca, ms.LT, 410, fmt=fp)
        y = ctx.project(cb, pos, fmt=fy)
        s = int(ms.to_numpy_u64(ctx.agg_sum(y))[0])
        assert_column(ctx, pos, want_pos, fp)
        assert_column(ctx, y, want_y, fy)
        assert s == want_sum
        for col in (y, pos, cb, ca):
            ctx.free(col)


# ------------------------------------------------------------------- errors

def test_errors_are_reported_not_trapped(ctx):
    assert ctx.get_error() == ms.MS_OK
    x = np.array([1, 2, 300], dtype=np.uint64)
    col, _ = gpu_col(ctx, x, ms.STATIC_BP, bw=8)
    assert ctx.get_error() == ms.MS_ERR_VALUE_TOO_WIDE
    ctx.free(col)

    d, _ = gpu_col(ctx, np.arange(100, dtype=np.uint64), ms.DYN_BP)
    p, _ = gpu_col(ctx, np.array([5, 100], dtype=np.uint64), ms.UNCOMPR)
    out = ctx.project(d, p)
    assert ctx.get_error() == ms.MS_ERR_OUT_OF_RANGE and ctx.last_error_info() == 100
    ctx.free(out)

    g, _ = gpu_col(ctx, np.array([0, 7], dtype=np.uint64), ms.UNCOMPR)
    v, _ = gpu_col(ctx, np.array([1, 1], dtype=np.uint64), ms.UNCOMPR)
    ctx.group_sum(g, v, 7)
    assert ctx.get_error() == ms.MS_ERR_OUT_OF_RANGE
    out = ctx.semijoin(v, g, 7)
    assert ctx.get_error() == ms.MS_ERR_OUT_OF_RANGE
    ctx.free(out)
    small = torch.empty(1, dtype=torch.int64, device=ctx.device)
    ctx.decompress(p, out=small)
    assert ctx.get_error() == ms.MS_ERR_INVALID_ARG
    for col in (v, g, p, d):
        ctx.free(col)

    x = synth.skewed_widths(3, 2048)
    buf = oracle.compress(oracle.DYN_BP, x).copy()
    buf[16] ^= 1
    bad = ctx.import_bytes(ms.DYN_BP, 2048, buf)
    assert ctx.get_error() == ms.MS_ERR_FORMAT
    ctx.free(bad)
    with pytest.raises(ms.MSError):
        ctx.compress(ms.as_device_u64(x, ctx.device), ms.STATIC_BP, 65)
    assert ctx.get_error() == ms.MS_OK


def test_arena_is_lifo_and_tracks_high_water(ctx):
    base, _ = ctx.arena_usage()
    ctx.reset_high_water()
    x = synth.skewed_widths(1, 10_000)
    a, _ = gpu_col(ctx, x, ms.DYN_BP)
    b, _ = gpu_col(ctx, x, ms.UNCOMPR)
    used, high = ctx.arena_usage()
    sa, sb = ctx.info(a)["size_bytes"], ctx.info(b)["size_bytes"]
    assert used - base >= sa + sb and high == used
    ctx.free(a)  # not the top: only marked
    assert ctx.arena_usage()[0] == used
    ctx.free(b)  # pops both
    assert ctx.arena_usage()[0] == base
    assert ctx.arena_usage()[1] == high


@pytest.mark.parametrize("fmt", [ms.DYN_BP, ms.DELTA_BP, ms.FOR_BP])
def test_block_outputs_stage_at_the_arena_end(fmt):
    """A block-format output waits in a stage taken from the arena's free end until
    the placement pass puts it behind its headers.  The high-water mark counts the
    stage beside the new column, the stage is released after every operator, and
    a column whose stage does not fit beside it is reported (MS_ERR_NOMEM) and
    published empty."""
    n = 500_000 + 37
    x = synth.skewed_widths(83, n)
    want = oracle.compress(fmt, x)
    size = want.nbytes
    payload = size - 16 * (n // 512) - 8 * (n % 512)
    with ms.Ctx(0, arena_bytes=4 * size + (1 << 20), max_rows=n) as big:
        base, _ = big.arena_usage()
        big.reset_high_water()
        col = big.compress(ms.as_device_u64(x, big.device), fmt)
        used, high = big.arena_usage()
        assert used - base == (size + 255) // 256 * 256
        assert high - base >= used - base + payload
        assert big.export_bytes(col).tobytes() == want.tobytes()
        for _ in range(6):  # each output's stage is released: repeated outputs fit
            tmp = big.calc(ms.ADD, col, None, 1, fmt=fmt)
            big.free(tmp)
        big.check(what="repeated staged outputs")
        big.free(col)
    arena = (size + size // 2 + 255) // 256 * 256  # the column alone fits, not beside its stage
    assert arena < size + payload
    with ms.Ctx(0, arena_bytes=arena, max_rows=n) as small:
        col = small.compress(ms.as_device_u64(x, small.device), fmt)
        assert small.get_error() == ms.MS_ERR_NOMEM
        assert small.info(col)["n"] == 0 and small.info(col)["size_bytes"] == 0
        small.free(col)
        assert small.get_error() == ms.MS_OK
        tiny = x[: 20_000]
        t = small.compress(ms.as_device_u64(tiny, small.device), fmt)
        small.check(what="stage released after a failed output")
        assert small.export_bytes(t).tobytes() == oracle.compress(fmt, tiny).tobytes()


@pytest.mark.parametrize("fmt", [ms.UNCOMPR, ms.DELTA_BP, ms.DYN_BP])
def test_select_and_semijoin_on_short_intermediates(ctx, fmt):
    """Operators on intermediates whose real length is far below the host-side
    bound must not read scratch past the real input (stale data from a larger
    earlier operator sits there)."""
    n = 40 * 4096 + 123
    x = synth.uniform(61, n, 0, 1000)
    cx, _ = gpu_col(ctx, x, ms.DYN_BP)
    big = ctx.select(cx, ms.LT, 900, fmt=fmt)  # leaves a large bitmap in scratch
    ctx.free(big)
    pos = ctx.select(cx, ms.LT, 37, fmt=fmt)  # ~3.7% of n, bound n
    want_pos = oracle.select(x, oracle.LT, 37)
    vals = ctx.project(cx, pos, fmt=fmt)
    want_vals = oracle.project(x, want_pos)
    q = ctx.select(vals, ms.GE, 20, fmt=fmt)
    assert_column(ctx, q, oracle.select(want_vals, oracle.GE, 20), fmt)
    keys_np = np.arange(0, 1000, 7, dtype=np.uint64)
    keys, _ = gpu_col(ctx, keys_np, ms.DELTA_BP)
    sj = ctx.semijoin(vals, keys, 1000, fmt=fmt)
    assert_column(ctx, sj, oracle.semijoin(want_vals, keys_np, 1000), fmt)
    for col in (sj, keys, q, vals, pos, cx):
        ctx.free(col)


@pytest.mark.parametrize("fmt", [ms.UNCOMPR, ms.DYN_BP, ms.STATIC_BP])
def test_arena_exhaustion_reports_nomem_and_leaves_an_empty_column(fmt):
    """A column that does not fit the arena is reported (MS_ERR_NOMEM) and
    published empty, so operators downstream never read outside the arena."""
    with ms.Ctx(0, arena_bytes=1 << 20, max_rows=1 << 20) as small:
        x = synth.skewed_widths(71, 600_000)  # > 1 MB in every format
        col = small.compress(ms.as_device_u64(x, small.device), fmt, 40 if fmt == ms.STATIC_BP else 0)
        assert small.get_error() == ms.MS_ERR_NOMEM
        assert small.info(col)["n"] == 0 and small.info(col)["size_bytes"] == 0
        s = small.agg_sum(col)
        pos = small.select(col, ms.LT, 5, fmt=fmt, bw=20 if fmt == ms.STATIC_BP else 0)
        assert int(ms.to_numpy_u64(s)[0]) == 0 and small.info(pos)["n"] == 0
        assert small.get_error() == ms.MS_OK
