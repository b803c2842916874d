"""Pins of the CPU oracle against facts fixed outside the oracle itself.

* hand-derived byte layouts (tests/golden/layout_examples.json),
* closed-form sizes (static BP: ceil(n*b/64)*8 bytes; block formats from the
  per-block width histogram),
* inverse identities (round trip for every format; FOR residual + reference,
  DELTA prefix sum + base),
* Table 1's printed maximum bit widths (tests/golden/table1.json),
* the paper's qualitative format outcomes (Sec. 5.1),
* numpy library routines for the operators (flatnonzero, take, wrapping sum,
  isin, add.at) and brute force on tiny inputs.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2004_09350_gb300 import synth

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _gold(name):
    with open(os.path.join(GOLD, name)) as f:
        return json.load(f)


def _hex(s):
    return bytes.fromhex(s.replace(" ", ""))


# ------------------------------------------------------------------ layout pins

def test_layout_static_bp_tail_hand_example():
    case = {c["name"]: c for c in _gold("layout_examples.json")["cases"]}["static_bp_tail_b3"]
    got = oracle.compress(oracle.STATIC_BP, case["values"], bw=3).tobytes()
    assert got == _hex(case["bytes_hex"])


def test_layout_static_bp_chunk_hand_example():
    x = np.arange(512, dtype=np.uint64) % 2
    assert oracle.compress(oracle.STATIC_BP, x, bw=1).tobytes() == b"\xaa" * 64


def test_layout_dyn_bp_hand_examples():
    x = np.arange(512, dtype=np.uint64) % 2
    want = _hex("0100000000000000 0000000000000000") + b"\xaa" * 64
    assert oracle.compress(oracle.DYN_BP, x).tobytes() == want

    x = np.zeros(513, dtype=np.uint64)
    x[83] = 15
    x[512] = 7
    payload = bytearray(256)
    payload[11] = 0xF0
    want = _hex("0400000000000000 0000000000000000") + bytes(payload) + _hex("0700000000000000")
    assert oracle.compress(oracle.DYN_BP, x).tobytes() == want


def test_layout_dyn_bp_two_blocks_hand_example():
    """Header chain (block 1's payload starts 8 words in) and a value that straddles
    two halfwords of its lane stream."""
    assert "dyn_bp_two_blocks_chain_and_straddle" in {c["name"] for c in _gold("layout_examples.json")["cases"]}
    x = np.zeros(1024, dtype=np.uint64)
    x[0], x[528], x[549], x[1023] = 1, 5, 7, 6
    p0, p1 = bytearray(64), bytearray(192)
    p0[0] = 0x01
    p1[2:4], p1[4:6], p1[68:70], p1[190:192] = b"\x05\x00", b"\x00\x80", b"\x03\x00", b"\x00\xc0"
    want = _hex("0100000000000000 0000000000000000 0308000000000000 0000000000000000") + bytes(p0) + bytes(p1)
    assert oracle.compress(oracle.DYN_BP, x).tobytes() == want
    np.testing.assert_array_equal(oracle.decompress(oracle.DYN_BP, x.size, oracle.compress(oracle.DYN_BP, x)), x)


def test_layout_for_bp_hand_example():
    x = 1000 + np.arange(512, dtype=np.uint64) % 4
    want = _hex("0200000000000000 e803000000000000") + b"\xe4" * 128
    assert oracle.compress(oracle.FOR_BP, x).tobytes() == want


def test_layout_delta_bp_hand_example():
    x = 5 + 3 * np.arange(512, dtype=np.uint64)
    want = _hex("0200000000000000 0500000000000000") + b"\xfc" + b"\xff" * 127
    assert oracle.compress(oracle.DELTA_BP, x).tobytes() == want


# --------------------------------------------------------------- closed forms

def _width(v: int) -> int:
    return int(v).bit_length()


@pytest.mark.parametrize("n", [0, 1, 63, 64, 511, 512, 513, 1000, 4097])
@pytest.mark.parametrize("b", [1, 3, 12, 31, 32, 33, 63, 64])
def test_static_bp_size_closed_form(n, b):
    x = synth.uniform(5, n, 0, 1 << b) if b < 64 else synth.splitmix64(5, n)
    assert oracle.size(oracle.STATIC_BP, x, bw=b) == -(-n * b // 64) * 8
    assert oracle.compress(oracle.STATIC_BP, x, bw=b).size == -(-n * b // 64) * 8


@pytest.mark.parametrize("fmt", [oracle.DYN_BP, oracle.FOR_BP, oracle.DELTA_BP])
@pytest.mark.parametrize("n", [0, 1, 511, 512, 513, 5000])
def test_block_format_size_from_width_histogram(fmt, n):
    x = synth.skewed_widths(9, n)
    nb, r = n // 512, n % 512
    total_bits = 0
    for k in range(nb):
        blk = [int(v) for v in x[512 * k: 512 * (k + 1)]]
        if fmt == oracle.DYN_BP:
            res = blk
        elif fmt == oracle.FOR_BP:
            res = [v - min(blk) for v in blk]
        else:
            res = [0] + [(blk[i] - blk[i - 1]) % 2**64 for i in range(1, 512)]
        total_bits += 512 * _width(max(res))
    assert oracle.size(fmt, x) == 16 * nb + total_bits // 8 + 8 * r


def test_dyn_bp_width_is_block_maximum_width():
    x = synth.skewed_widths(3, 512 * 40)
    widths = oracle.block_widths(oracle.DYN_BP, x)
    want = [_width(int(x[512 * k: 512 * (k + 1)].max())) for k in range(40)]
    assert list(widths) == want
    assert set(want) <= set(synth.WIDTH_CHOICES)


def test_delta_of_constant_gap_has_gap_width():
    for gap in (1, 2, 3, 1000, 2**40 + 1):
        x = 7 + gap * np.arange(512 * 3 + 5, dtype=np.uint64)
        assert list(oracle.block_widths(oracle.DELTA_BP, x)) == [_width(gap)] * 3
        assert oracle.size(oracle.DELTA_BP, x) == 16 * 3 + 3 * 64 * _width(gap) + 8 * 5


def test_for_of_narrow_range_has_range_width():
    x = synth.uniform(4, 512 * 4, 2**62, 2**62 + 64)
    x[0] = 2**62
    x[512:1024] = 2**62 + 5 + (np.arange(512, dtype=np.uint64) % 9)
    w = oracle.block_widths(oracle.FOR_BP, x)
    assert w[1] == _width(8)
    assert all(v <= 6 for v in w)


# ----------------------------------------------------------- inverse identities

EDGE_NS = [0, 1, 15, 16, 511, 512, 513, 1023, 1024, 4097]


def _edge_column(n, b, seed=1):
    if b == 0:
        return np.zeros(n, dtype=np.uint64)
    x = synth.splitmix64(seed, n) >> np.uint64(64 - b)
    if n:
        x[n // 2] |= np.uint64(1) << np.uint64(b - 1)
    return x


@pytest.mark.parametrize("fmt", range(5))
@pytest.mark.parametrize("n", EDGE_NS)
@pytest.mark.parametrize("b", [0, 1, 31, 32, 33, 63, 64])
def test_round_trip_identity(fmt, n, b):
    x = _edge_column(n, b)
    bw = max(b, 1)
    buf = oracle.compress(fmt, x, bw=bw)
    assert oracle.size(fmt, x, bw=bw) == buf.size
    np.testing.assert_array_equal(oracle.decompress(fmt, n, buf, bw=bw), x)


def test_round_trip_large_mixed():
    n = (1 << 20) + 7
    cols = [synth.skewed_widths(1, n), synth.sorted_gaps(2, n), synth.table1_column("C3", n)]
    for x in cols:
        for fmt in range(5):
            bw = max(1, _width(int(x.max())))
            buf = oracle.compress(fmt, x, bw=bw)
            np.testing.assert_array_equal(oracle.decompress(fmt, n, buf, bw=bw), x)


def _payload_residuals(buf, n):
    """Read residuals and references straight from the bytes with numpy bit ops."""
    nb = n // 512
    hdr = np.frombuffer(buf[: 16 * nb].tobytes(), dtype="<u8").reshape(nb, 2)
    payload = buf[16 * nb:]
    out, refs = [], []
    for k in range(nb):
        w0, ref = int(hdr[k, 0]), int(hdr[k, 1])
        b, off = w0 & 0xFF, w0 >> 8
        blk = np.frombuffer(payload[8 * off: 8 * off + 64 * b].tobytes(), dtype="<u2")
        hw = blk.reshape(b, 32) if b else np.zeros((0, 32), dtype="<u2")
        bits = np.unpackbits(hw.T.copy().view(np.uint8), bitorder="little").reshape(32, 16 * b)
        vals = []
        for j in range(32):
            for kk in range(16):
                chunk = bits[j, kk * b:(kk + 1) * b]
                vals.append(int(sum(int(c) << s for s, c in enumerate(chunk))))
        out.append(vals)
        refs.append(ref)
    return out, refs


def test_for_inverse_identity_from_bytes():
    x = synth.table1_column("C3", 512 * 3)
    buf = oracle.compress(oracle.FOR_BP, x)
    res, refs = _payload_residuals(buf, x.size)
    for k in range(3):
        blk = [int(v) for v in x[512 * k: 512 * (k + 1)]]
        assert refs[k] == min(blk)
        assert [refs[k] + r for r in res[k]] == blk


def test_delta_inverse_identity_from_bytes():
    x = synth.sorted_gaps(8, 512 * 3)
    buf = oracle.compress(oracle.DELTA_BP, x)
    res, refs = _payload_residuals(buf, x.size)
    for k in range(3):
        blk = [int(v) for v in x[512 * k: 512 * (k + 1)]]
        assert refs[k] == blk[0] and res[k][0] == 0
        assert list(np.cumsum([refs[k]] + res[k][1:], dtype=object)) == blk


def test_bad_header_is_rejected():
    x = synth.skewed_widths(2, 1024)
    buf = oracle.compress(oracle.DYN_BP, x).copy()
    buf[16] ^= 0x01  # block 1's width no longer matches the running offset
    with pytest.raises(oracle.OracleError):
        oracle.decompress(oracle.DYN_BP, 1024, buf)
    with pytest.raises(oracle.OracleError):
        oracle.compress(oracle.STATIC_BP, [8], bw=3)  # 8 needs 4 bits


# ------------------------------------------------------------- paper outcomes

def test_table1_max_bit_widths():
    gold = _gold("table1.json")["max_bit_width"]
    for name, want in gold.items():
        x = synth.table1_column(name, 1 << 20)
        assert oracle.bitwidth(int(x.max())) == want, name


def test_paper_best_formats_by_size():
    # Sec. 5.1: static BP for C1 (small values), SIMD-BP512 for C2 (outliers),
    # FOR+BP for C3 (narrow range of huge values), DELTA+BP for C4 (sorted).
    n = 1 << 20
    best = {c: oracle.best_format_by_size(synth.table1_column(c, n)) for c in ("C1", "C2", "C3", "C4")}
    assert best == {"C1": "static_bp", "C2": "dyn_bp", "C3": "for_bp", "C4": "delta_bp"}
    s1 = oracle.sizes_all_formats(synth.table1_column("C1", n))
    assert s1["static_bp"] == n * 6 // 8  # compression to 6/64 of 8n bytes
    # select positions are sorted: DELTA+BP is the best output format (Sec. 5.1)
    x = synth.table1_point_select_variant("C1", n)
    pos = oracle.select(x, oracle.EQ, 0)
    assert 0.89 < pos.size / n < 0.91
    assert oracle.best_format_by_size(pos) == "delta_bp"


# ------------------------------------------------------------------- operators

CMPS = [(oracle.EQ, np.equal), (oracle.NE, np.not_equal), (oracle.LT, np.less),
        (oracle.LE, np.less_equal), (oracle.GT, np.greater), (oracle.GE, np.greater_equal)]


@pytest.mark.parametrize("cmp,fn", CMPS)
def test_select_matches_flatnonzero(cmp, fn):
    x = synth.uniform(3, 5000, 0, 100)
    for c in (0, 1, 50, 99, 100, 2**64 - 1):
        got = oracle.select(x, cmp, c)
        np.testing.assert_array_equal(got, np.flatnonzero(fn(x, np.uint64(c))).astype(np.uint64))


def test_select_between_and_empty():
    x = synth.uniform(4, 3000, 0, 1000)
    got = oracle.select(x, oracle.BETWEEN, 100, 200)
    np.testing.assert_array_equal(got, np.flatnonzero((x >= 100) & (x <= 200)).astype(np.uint64))
    assert oracle.select(np.zeros(0, np.uint64), oracle.LT, 5).size == 0
    assert oracle.select(x, oracle.BETWEEN, 200, 100).size == 0


def test_select_brute_force_tiny_exhaustive():
    x = np.array([3, 0, 7, 7, 1, 2**64 - 1, 5], dtype=np.uint64)
    for cmp in range(6):
        for c in range(0, 9):
            want = [i for i, v in enumerate(x.tolist()) if
                    [v == c, v != c, v < c, v <= c, v > c, v >= c][cmp]]
            assert oracle.select(x, cmp, c).tolist() == want


def test_project_matches_take():
    d = synth.splitmix64(5, 10000)
    pos = np.sort(synth.uniform(6, 3000, 0, 10000))
    np.testing.assert_array_equal(oracle.project(d, pos), np.take(d, pos.astype(np.int64)))
    with pytest.raises(oracle.OracleError):
        oracle.project(d, np.array([10000], dtype=np.uint64))
    assert oracle.project(d, np.zeros(0, np.uint64)).size == 0


def test_calc_wraps_modulo_2_64():
    a, b = synth.splitmix64(1, 2000), synth.splitmix64(2, 2000)
    with np.errstate(over="ignore"):
        np.testing.assert_array_equal(oracle.calc(oracle.ADD, a, b), a + b)
        np.testing.assert_array_equal(oracle.calc(oracle.SUB, a, b), a - b)
        np.testing.assert_array_equal(oracle.calc(oracle.MUL, a, b), a * b)
        np.testing.assert_array_equal(oracle.calc(oracle.MUL, a, c=15), a * np.uint64(15))
    assert int(oracle.calc(oracle.MUL, [2**63], [2])[0]) == 0


def test_agg_sum_wraps_and_matches_numpy():
    x = synth.splitmix64(3, 100001)
    assert oracle.agg_sum(x) == int(np.add.reduce(x, dtype=np.uint64))
    assert oracle.agg_sum(x) == sum(int(v) for v in x) % 2**64
    assert oracle.agg_sum(np.zeros(0, np.uint64)) == 0


def test_group_sum_matches_add_at():
    g = synth.uniform(1, 50000, 0, 105)
    v = synth.splitmix64(2, 50000)
    want = np.zeros(105, dtype=np.uint64)
    np.add.at(want, g.astype(np.int64), v)
    np.testing.assert_array_equal(oracle.group_sum(g, v, 105), want)
    with pytest.raises(oracle.OracleError):
        oracle.group_sum([105], [1], 105)


def test_semijoin_matches_isin():
    probe = synth.uniform(1, 40000, 0, 3000)
    keys = synth.uniform(2, 500, 0, 3000)
    got = oracle.semijoin(probe, keys, 3000)
    np.testing.assert_array_equal(got, np.flatnonzero(np.isin(probe, keys)).astype(np.uint64))
    dup = np.concatenate([keys, keys])
    np.testing.assert_array_equal(oracle.semijoin(probe, dup, 3000), got)
    assert oracle.semijoin(probe, np.zeros(0, np.uint64), 3000).size == 0
    with pytest.raises(oracle.OracleError):
        oracle.semijoin(probe, [3000], 3000)


# ------------------------------------------------------------------ RLE pins

def _rle_case_values(case):
    if "values" in case:
        return np.array(case["values"], dtype=np.uint64)
    return np.concatenate([np.full(k, v, dtype=np.uint64) for v, k in case["values_rle"]])


@pytest.mark.parametrize("name", ["rle_three_runs", "rle_run_across_a_block_boundary", "rle_run_starting_at_a_block"])
def test_layout_rle_hand_examples(name):
    case = {c["name"]: c for c in _gold("layout_examples.json")["cases"]}[name]
    x = _rle_case_values(case)
    assert oracle.compress(oracle.RLE, x).tobytes() == _hex(case["bytes_hex"])
    raw = np.frombuffer(_hex(case["bytes_hex"]), dtype=np.uint8)
    np.testing.assert_array_equal(oracle.decompress(oracle.RLE, x.size, raw), x)


def _rle_parts(buf, n):
    """Run values, run ends and directory read straight from the bytes."""
    w = np.frombuffer(buf.tobytes(), dtype="<u8")
    nch = -(-n // 512)
    R = (w.size - nch) // 2
    return w[:R], w[R:2 * R], w[2 * R:]


def _runny(seed, n, mean_run):
    """Values drawn with runs of geometric length (mean `mean_run`)."""
    rng = np.random.default_rng(seed)
    lens = rng.geometric(1.0 / mean_run, size=n + 1)
    vals = rng.integers(0, 6, size=lens.size).astype(np.uint64)  # few values: equal neighbours merge
    return np.repeat(vals, lens)[:n]


@pytest.mark.parametrize("n", [0, 1, 2, 511, 512, 513, 1024, 1500, 4097])
@pytest.mark.parametrize("mean_run", [1, 3, 40, 700])
def test_rle_bytes_decode_with_numpy_repeat(n, mean_run):
    """The bytes decode by np.repeat(values, diff(ends)); the size is the closed form
    16 * (1 + number of changes) + 8 * ceil(n / 512); the directory entry of block g
    is the run that holds value 512 g (searchsorted over the ends)."""
    x = _runny(n * 7 + mean_run, n, mean_run)
    buf = oracle.compress(oracle.RLE, x)
    runs = 1 + int(np.count_nonzero(np.diff(x))) if n else 0
    assert buf.size == 16 * runs + 8 * (-(-n // 512)) == oracle.size(oracle.RLE, x)
    vals, ends, dirs = _rle_parts(buf, n)
    assert vals.size == runs
    lens = np.diff(np.concatenate([[0], ends]).astype(np.int64))
    assert (lens > 0).all()
    np.testing.assert_array_equal(np.repeat(vals, lens), x)
    np.testing.assert_array_equal(dirs, np.searchsorted(ends, 512 * np.arange(dirs.size), side="right"))
    # the run-weighted sum of the values is the column sum (mod 2^64)
    assert int((vals * lens.astype(np.uint64)).sum(dtype=np.uint64)) == int(x.sum(dtype=np.uint64))
    np.testing.assert_array_equal(oracle.decompress(oracle.RLE, n, buf), x)


def test_rle_special_cases():
    x = np.full(1000, 42, dtype=np.uint64)  # one run
    assert oracle.compress(oracle.RLE, x).view("<u8").tolist() == [42, 1000, 0, 0]
    x = np.arange(600, dtype=np.uint64)  # every value its own run
    vals, ends, dirs = _rle_parts(oracle.compress(oracle.RLE, x), 600)
    assert vals.tolist() == list(range(600)) and ends.tolist() == list(range(1, 601)) and dirs.tolist() == [0, 512]
    assert oracle.compress(oracle.RLE, np.zeros(0, dtype=np.uint64)).size == 0


def test_rle_corrupt_columns_are_rejected():
    x = _runny(3, 1500, 40)
    buf = oracle.compress(oracle.RLE, x)
    vals, ends, dirs = _rle_parts(buf, x.size)
    R = vals.size
    bad = buf.view("<u8").copy()
    bad[R + R - 1] = x.size - 1  # the last run must end at n
    with pytest.raises(oracle.OracleError):
        oracle.decompress(oracle.RLE, x.size, bad.view(np.uint8))
    bad = buf.view("<u8").copy()
    bad[R + 1] = bad[R]  # an empty run
    with pytest.raises(oracle.OracleError):
        oracle.decompress(oracle.RLE, x.size, bad.view(np.uint8))
    bad = buf.view("<u8").copy()
    bad[2 * R + 1] += 1  # block 1's directory entry names the wrong run
    with pytest.raises(oracle.OracleError):
        oracle.decompress(oracle.RLE, x.size, bad.view(np.uint8))
    with pytest.raises(oracle.OracleError):
        oracle.decompress(oracle.RLE, x.size, buf[:-8])  # not 16 R + 8 nch bytes


# ----------------------------------------------- FOR / DELTA cascaded with static BP

@pytest.mark.parametrize("fmt,base", [(oracle.FOR_STATIC_BP, oracle.FOR_BP), (oracle.DELTA_STATIC_BP, oracle.DELTA_BP)])
def test_static_cascade_equals_block_format_at_its_natural_width(fmt, base):
    """When every block's residuals need exactly b bits, the cascade with static BP at
    width b writes the same bytes as the cascade with dynamic BP."""
    x = (1000 + np.arange(3 * 512 + 100, dtype=np.uint64) % 4) if base == oracle.FOR_BP else \
        (5 + 3 * np.arange(3 * 512 + 100, dtype=np.uint64))
    b = int(oracle.block_widths(base, x).max())
    assert (oracle.block_widths(base, x) == b).all()
    assert oracle.compress(fmt, x, bw=b).tobytes() == oracle.compress(base, x).tobytes()


@pytest.mark.parametrize("fmt", [oracle.FOR_STATIC_BP, oracle.DELTA_STATIC_BP])
@pytest.mark.parametrize("n", [0, 1, 511, 512, 513, 1500, 4097])
def test_static_cascade_bytes_size_and_residuals(fmt, n):
    """Every header carries width bw at offset 8*bw*k; the residuals read from the bytes
    with numpy bit operations give the values back (reference + residual for FOR, the
    prefix sum from the reference for DELTA); size 16 nb + 64 bw nb + 8 r."""
    x = synth.sorted_gaps(91, n) if fmt == oracle.DELTA_STATIC_BP else synth.table1_column("C3", n)
    need = int(oracle.block_widths(oracle.DELTA_BP if fmt == oracle.DELTA_STATIC_BP else oracle.FOR_BP, x).max()) \
        if n >= 512 else 1
    bw = need + 3
    buf = oracle.compress(fmt, x, bw=bw)
    nb, r = n // 512, n % 512
    assert buf.size == 16 * nb + 64 * bw * nb + 8 * r == oracle.size(fmt, x, bw=bw)
    hdr = np.frombuffer(buf[: 16 * nb].tobytes(), dtype="<u8").reshape(nb, 2) if nb else np.zeros((0, 2), np.uint64)
    assert [int(w) & 0xFF for w in hdr[:, 0]] == [bw] * nb
    assert [int(w) >> 8 for w in hdr[:, 0]] == [8 * bw * k for k in range(nb)]
    res, refs = _payload_residuals(buf, n)
    for k in range(nb):
        blk = [int(v) for v in x[512 * k: 512 * (k + 1)]]
        if fmt == oracle.FOR_STATIC_BP:
            assert refs[k] == min(blk) and [refs[k] + q for q in res[k]] == blk
        else:
            assert refs[k] == blk[0] and res[k][0] == 0
            assert list(np.cumsum([refs[k]] + res[k][1:], dtype=object)) == blk
    np.testing.assert_array_equal(oracle.decompress(fmt, n, buf, bw=bw), x)


def test_static_cascade_width_limits():
    x = synth.sorted_gaps(92, 2048)
    need = int(oracle.block_widths(oracle.DELTA_BP, x).max())
    oracle.compress(oracle.DELTA_STATIC_BP, x, bw=need)
    with pytest.raises(oracle.OracleError):
        oracle.compress(oracle.DELTA_STATIC_BP, x, bw=need - 1)
    y = synth.table1_column("C3", 2048)  # FOR residuals below 2^6
    with pytest.raises(oracle.OracleError):
        oracle.compress(oracle.FOR_STATIC_BP, y, bw=5)
    buf = oracle.compress(oracle.FOR_STATIC_BP, y, bw=6)
    with pytest.raises(oracle.OracleError):  # read back at another width: headers disagree
        oracle.decompress(oracle.FOR_STATIC_BP, y.size, buf, bw=7)
