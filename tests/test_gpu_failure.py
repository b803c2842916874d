"""Failure detection on the GPU without a fault: a device wait that nothing ever
satisfies gives up after its iteration limit with MS_ERR_TIMEOUT, the error word
clears on read, and the same context then computes correct results."""
import numpy as np
import pytest

import oracle
from paper_2004_09350_gb300 import morphstore as ms
from paper_2004_09350_gb300 import synth

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_and_the_context_survives():
    ctx = ms.Ctx(0, arena_bytes=1 << 26, max_rows=1 << 16)
    ctx.selftest_wait_timeout()
    assert ctx.get_error() == ms.MS_ERR_TIMEOUT
    assert ctx.last_error_info() == 1  # the waiting tile
    assert ctx.get_error() == ms.MS_OK  # read and cleared
    x = synth.uniform(5, 9000, 0, 1 << 20)
    col = ctx.compress(ms.as_device_u64(x, ctx.device), ms.DYN_BP)
    pos = ctx.select(col, ms.LT, 1 << 19, fmt=ms.DELTA_BP)
    got = int(ms.to_numpy_u64(ctx.agg_sum(ctx.project(col, pos)))[0])
    ctx.check(what="after the timeout")
    assert got == oracle.agg_sum(oracle.project(x, oracle.select(x, oracle.LT, 1 << 19)))
    ctx.close()


def test_device_errors_are_sticky_until_read():
    ctx = ms.Ctx(0, arena_bytes=1 << 26, max_rows=1 << 16)
    x = synth.uniform(6, 1000, 0, 100)
    col = ctx.compress(ms.as_device_u64(x, ctx.device), ms.UNCOMPR)
    bad = ctx.compress(ms.as_device_u64(np.array([5, 2000], dtype=np.uint64), ctx.device), ms.UNCOMPR)
    out = ctx.project(col, bad)  # position 2000 is out of range
    ctx.selftest_wait_timeout()  # a later error does not overwrite the first
    assert ctx.get_error() == ms.MS_ERR_OUT_OF_RANGE
    assert ctx.last_error_info() == 2000
    assert ctx.get_error() == ms.MS_OK
    for c in (out, bad, col):
        ctx.free(c)
    ctx.close()
