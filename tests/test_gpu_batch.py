"""GPU parity of batched fragments (ms_batch_*): one persistent launch over many
select -> project -> agg_sum fragments against the oracle's three operators.

Sums modulo 2^64 are exact, so the bar is bit-exact for every fragment, every
kernel configuration, one launch per fragment, sub-ranges and CUDA graph replay.
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
    c = ms.Ctx(0, arena_bytes=4 << 30, max_rows=1 << 22)
    yield c
    c.close()


def oracle_sum(x, y, cmp, c1, c2):
    """The fragment as the oracle's select -> project -> agg_sum."""
    pos = oracle.select(x, cmp, c1, c2)
    return oracle.agg_sum(oracle.project(y, pos))


def col(ctx, a, fmt):
    bw = max(1, int(a.max()).bit_length()) if a.size else 1
    return ctx.compress(ms.as_device_u64(a, ctx.device), fmt, bw if fmt == ms.STATIC_BP else 0)


def wide(seed, n, b):
    x = synth.splitmix64(seed, n) >> np.uint64(64 - b)
    if n:
        x[n // 2] |= np.uint64(1) << np.uint64(b - 1)
    return x


def small_fragments():
    """Ragged lengths (empty, one value, chunk edges, several tiles), every format
    for x and y, all predicates, widths above the staging slot (48 and 64 bits)."""
    specs = synth.batch_fragments(11, 48, lo_log2=0, hi_log2=15)
    for i, n in enumerate([0, 1, 511, 512, 513, 1023, 1537, 4096 * 3 + 5, 0, 700]):
        specs[i]["n"] = n
    frags = []
    for i, sp in enumerate(specs):
        frags.append((synth.batch_x(sp), synth.batch_y(sp), sp["cmp"], sp["c1"], sp["c2"]))
    for i, (n, b) in enumerate([(2000, 48), (5000, 64), (513, 41)]):
        x = wide(100 + i, n, b)
        y = wide(200 + i, n, 64)
        frags.append((x, y, ms.LT, int(x[n // 3]), 0))
    return frags


@pytest.fixture(scope="module")
def batch(ctx):
    frags = small_fragments()
    xs, ys = [], []
    for i, (x, y, *_) in enumerate(frags):
        xs.append(col(ctx, x, FMTS[i % 5]))
        ys.append(col(ctx, y, FMTS[(i // 5 + i) % 5]))
    b = ms.Batch(ctx, xs, ys, [f[2] for f in frags], [f[3] for f in frags], [f[4] for f in frags])
    want = np.array([oracle_sum(*f) for f in frags], dtype=np.uint64)
    yield b, want, frags
    b.close()


def run(ctx, b, **kw):
    sums = torch.full((b.n,), 7, dtype=torch.int64, device=ctx.device)
    b.run(sums, **kw)
    ctx.check(what="batch")
    return ms.to_numpy_u64(sums)


def test_batch_matches_oracle(ctx, batch):
    b, want, frags = batch
    info = b.info()
    assert info["rows"] == sum(f[0].size for f in frags)
    assert info["chunks"] == sum((f[0].size + 511) // 512 for f in frags)
    np.testing.assert_array_equal(run(ctx, b), want)


CONFIGS = [(w, d, t, k, c, s) for (w, d, c, s) in ms.BATCH_VARIANTS
           for t, k in ((max(8, w), 0), (64, 1), (1024, 0))]


@pytest.mark.parametrize("cfg", CONFIGS, ids=lambda c: "w%d-d%d-t%d-k%d-c%d-s%d" % c)
def test_every_configuration_gives_the_same_bits(ctx, batch, cfg):
    b, want, _ = batch
    np.testing.assert_array_equal(run(ctx, b, cfg=cfg), want)


def test_one_launch_per_fragment(ctx, batch):
    b, want, _ = batch
    np.testing.assert_array_equal(run(ctx, b, per_fragment=True), want)


def test_sub_range_accumulates_and_leaves_the_rest(ctx, batch):
    b, want, _ = batch
    sums = torch.full((b.n,), 7, dtype=torch.int64, device=ctx.device)
    f0, f1 = 5, 31
    b.run(sums, f0=f0, f1=f1)
    b.run(sums, f0=f0, f1=f1, zero=False, cfg=(4, 2, 16, 1, 1, 0))
    ctx.check(what="batch")
    got = ms.to_numpy_u64(sums)
    with np.errstate(over="ignore"):
        np.testing.assert_array_equal(got[f0:f1], want[f0:f1] * np.uint64(2))
    assert (got[:f0] == 7).all() and (got[f1:] == 7).all()


def test_graph_replay_is_identical(ctx, batch):
    b, want, _ = batch
    sums = torch.zeros(b.n, dtype=torch.int64, device=ctx.device)
    for per_fragment in (False, True):
        g = b.graph(sums, cfg=(8, 4, 32, 0, 0, 0) if per_fragment else (16, 2, 64, 0, 0, 1),
                    per_fragment=per_fragment)
        for _ in range(3):
            sums.fill_(-1)
            g.launch()
            ctx.check(what="graph")
            np.testing.assert_array_equal(ms.to_numpy_u64(sums), want)
        g.close()


def test_operator_outputs_bind_by_device_metadata(ctx):
    """Columns whose lengths exist only on the device (operator outputs)."""
    n = 9000
    a = synth.uniform(3, n, 0, 1 << 20)
    bcol = synth.uniform(4, n, 0, 1 << 30)
    ca, cb = col(ctx, a, ms.DYN_BP), col(ctx, bcol, ms.FOR_BP)
    pos = ctx.select(ca, ms.LT, 1 << 19, fmt=ms.DELTA_BP)
    xa = ctx.project(ca, pos, fmt=ms.DYN_BP)
    yb = ctx.project(cb, pos, fmt=ms.DELTA_BP)
    bt = ms.Batch(ctx, [xa, ca], [yb, cb], [ms.GE, ms.BETWEEN], [1 << 18, 1000], [0, 1 << 19])
    got = run(ctx, bt)
    p = oracle.select(a, ms.LT, 1 << 19)
    xa_h, yb_h = oracle.project(a, p), oracle.project(bcol, p)
    want = [oracle_sum(xa_h, yb_h, ms.GE, 1 << 18, 0), oracle_sum(a, bcol, ms.BETWEEN, 1000, 1 << 19)]
    np.testing.assert_array_equal(got, np.array(want, dtype=np.uint64))
    bt.close()
    for c in (yb, xa, pos, cb, ca):
        ctx.free(c)


def test_all_empty_fragments_give_zero(ctx):
    e = col(ctx, np.zeros(0, dtype=np.uint64), ms.DYN_BP)
    bt = ms.Batch(ctx, [e, e], [e, e], [ms.LE, ms.NE], [5, 5])
    np.testing.assert_array_equal(run(ctx, bt), np.zeros(2, dtype=np.uint64))
    bt.close()
    ctx.free(e)


def test_errors_are_reported(ctx, batch):
    b, _, _ = batch
    a = col(ctx, np.arange(10, dtype=np.uint64), ms.UNCOMPR)
    c = col(ctx, np.arange(11, dtype=np.uint64), ms.UNCOMPR)
    with pytest.raises(ms.MSError) as e:
        ms.Batch(ctx, [a], [c], [ms.LT], [3])
    assert e.value.code == ms.MS_ERR_INVALID_ARG
    with pytest.raises(ms.MSError):
        ms.Batch(ctx, [a], [a], [9], [3])
    sums = torch.zeros(b.n, dtype=torch.int64, device=ctx.device)
    for cfg in ((6, 3, 32, 0, 0, 0), (8, 5, 32, 0, 0, 0), (8, 4, 4, 0, 0, 0), (8, 3, 24, 0, 0, 0),
                (8, 3, 2048, 0, 0, 0), (8, 3, 32, 0, 2, 0), (16, 2, 8, 0, 0, 1), (16, 3, 64, 0, 0, 1),
                (8, 2, 64, 0, 1, 1), (8, 2, 64, 0, 0, 3), (4, 2, 64, 0, 0, 2), (8, 2, 64, 0, 1, 2)):
        with pytest.raises(ms.MSError) as e:
            b.run(sums, cfg=cfg)
        assert e.value.code == ms.MS_ERR_INVALID_ARG
    with pytest.raises(ms.MSError):
        b.run(sums, f0=3, f1=b.n + 1)
    ctx.free(c)
    ctx.free(a)


def test_batch_at_scale_sampled_against_oracle(ctx):
    """512 fragments, lengths log-uniform in [2^10, 2^20] (the batched workload's
    distribution at a smaller upper end), formats cycling; 24 fragments checked
    against the oracle, every fragment against one launch per fragment."""
    specs = synth.batch_fragments(23, 512, lo_log2=10, hi_log2=20)
    c = ms.Ctx(0, arena_bytes=2 << 30, max_rows=1 << 20)
    xs, ys = [], []
    for i, sp in enumerate(specs):
        xs.append(col_t(c, synth.batch_x_torch(sp, c.device), FMTS[(i + 1) % 5], sp["bx"]))
        ys.append(col_t(c, synth.batch_y_torch(sp, c.device), FMTS[(3 * i) % 5], None))
    bt = ms.Batch(c, xs, ys, [s["cmp"] for s in specs], [s["c1"] for s in specs], [s["c2"] for s in specs])
    got = run(c, bt)
    each = run(c, bt, per_fragment=True, cfg=(4, 2, 8, 0, 1, 0))
    stat = run(c, bt, cfg=(16, 2, 16, 0, 0, 1))
    np.testing.assert_array_equal(got, stat)
    np.testing.assert_array_equal(got, each)
    rng = np.random.default_rng(0)
    order = np.argsort([s["n"] for s in specs])
    sample = set(order[-8:].tolist()) | set(order[:4].tolist()) | set(rng.choice(512, 12, replace=False).tolist())
    for f in sorted(sample):
        sp = specs[f]
        assert got[f] == oracle_sum(synth.batch_x(sp), synth.batch_y(sp), sp["cmp"], sp["c1"], sp["c2"]), f
    bt.close()
    c.close()


def col_t(ctx, t, fmt, bits):
    bw = bits if bits is not None else max(1, int(t.max().item()).bit_length())
    return ctx.compress(t, fmt, bw if fmt == ms.STATIC_BP else 0)
