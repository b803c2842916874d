"""The algorithmic byte counts behind the bench's roofline, on the CPU: block widths
and touched-block bytes against brute force, and against the oracle's compressed
sizes when every position is touched."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402
import oracle  # noqa: E402
from paper_2004_09350_gb300 import synth  # noqa: E402


def brute_widths(x, delta=False):
    out = []
    for g in range(x.size // 512):
        blk = [int(v) for v in x[512 * g: 512 * g + 512]]
        vals = [(blk[i] - blk[i - 1]) % 2**64 for i in range(1, 512)] if delta else blk
        out.append(max(vals).bit_length())
    return out


def test_block_widths_match_brute_force():
    x = synth.skewed_widths(5, 7 * 512 + 100, widths=(0, 1, 13, 40, 64))
    assert list(bench.block_widths(x)) == brute_widths(x)
    k = synth.sorted_gaps(6, 5 * 512 + 3)
    assert list(bench.block_widths(k, delta=True)) == brute_widths(k, delta=True)
    u = synth.uniform(7, 3 * 512, 0, 1000)  # unsorted: deltas wrap modulo 2^64
    assert list(bench.block_widths(u, delta=True)) == brute_widths(u, delta=True)


def test_touched_bytes_match_brute_force():
    n = 9 * 512 + 77
    x = synth.skewed_widths(8, n)
    w = bench.block_widths(x)
    pos = np.unique(synth.uniform(9, 300, 0, n))
    blocks = sorted({int(p) // 512 for p in pos if p < 9 * 512})
    sectors = {(8 * (int(p) - 9 * 512)) // 32 for p in pos if p >= 9 * 512}
    want = sum(16 + 64 * int(w[g]) for g in blocks) + 32 * len(sectors)
    assert bench.touched_bytes_dyn(w, n, pos) == want
    k = synth.sorted_gaps(10, n)
    wk = bench.block_widths(k, delta=True)
    assert bench.touched_bytes_delta(wk, pos) == sum(64 * int(wk[g]) + 16 for g in blocks)


def test_touching_every_row_costs_the_compressed_size():
    n = 6 * 512 + 64  # remainder of 64 values = 16 whole 32-byte sectors
    x = synth.skewed_widths(11, n)
    every = np.arange(n, dtype=np.uint64)
    assert bench.touched_bytes_dyn(bench.block_widths(x), n, every) == oracle.compress(oracle.DYN_BP, x).size
    k = synth.sorted_gaps(12, 6 * 512)
    assert bench.touched_bytes_delta(bench.block_widths(k, delta=True), every[: k.size]) == \
        oracle.compress(oracle.DELTA_BP, k).size
