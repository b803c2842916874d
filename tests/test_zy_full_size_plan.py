"""The default bench plan at its full size (two 2^28-row columns, the bench's own
seeded inputs, arena and formats: X dynamic BP, K DELTA, P DELTA, X' dynamic BP,
K' DELTA, Y dynamic BP), checked element by element against the oracle's operators
run on the uncompressed columns: every position, projected value and product, and
the sum.  The oracle's operators are single C loops, quick at this size; the GPU
intermediates are decompressed on the GPU for the comparison, so the oracle's
bit-level codec is not needed here (the smaller parity tests compare bytes)."""
import numpy as np
import pytest
import torch

import bench
import oracle
from paper_2004_09350_gb300 import morphstore as ms

pytestmark = pytest.mark.gpu


def test_full_size_plan_matches_the_oracle():
    n = 1 << 28
    x, k, c = bench.make_inputs(n, 2020, 0.1)
    dev = torch.device("cuda", 0)
    ctx = ms.Ctx(0, arena_bytes=int(2.5 * 8 * n) + (1 << 30), max_rows=n)
    try:
        cx = ctx.compress(ms.as_device_u64(x, dev), ms.DYN_BP)
        ck = ctx.compress(ms.as_device_u64(k, dev), ms.DELTA_BP)
        pos = ctx.select(cx, ms.LT, c, fmt=ms.DELTA_BP)
        xp = ctx.project(cx, pos, fmt=ms.DYN_BP)
        kp = ctx.project(ck, pos, fmt=ms.DELTA_BP)
        y = ctx.calc(ms.MUL, xp, kp, fmt=ms.DYN_BP)
        got_sum = int(ms.to_numpy_u64(ctx.agg_sum(y))[0])
        ctx.check(what="full-size plan")

        want_pos = oracle.select(x, oracle.LT, c)
        assert 0.05 < want_pos.size / n < 0.15
        np.testing.assert_array_equal(ms.to_numpy_u64(ctx.decompress(pos)), want_pos)
        want_xp = oracle.project(x, want_pos)
        want_kp = oracle.project(k, want_pos)
        np.testing.assert_array_equal(ms.to_numpy_u64(ctx.decompress(xp)), want_xp)
        np.testing.assert_array_equal(ms.to_numpy_u64(ctx.decompress(kp)), want_kp)
        want_y = oracle.calc(oracle.MUL, want_xp, want_kp)
        np.testing.assert_array_equal(ms.to_numpy_u64(ctx.decompress(y)), want_y)
        assert got_sum == oracle.agg_sum(want_y)
        ctx.check(what="decompress")
    finally:
        ctx.close()
