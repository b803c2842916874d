"""Star-schema plan through the C ABI against the same plan on the oracle.

The plan is two dimension selects, two semi-joins into the fact table, range
selects on discount and quantity, projects, calc and a 105-group sum.  It runs
with compressed intermediates, with uncompressed ones, and with uncompressed
base columns.  The group sums must equal the oracle's bit for bit.
"""
import numpy as np
import pytest

import oracle
from paper_2004_09350_gb300 import morphstore as ms
from paper_2004_09350_gb300 import plans, synth

pytestmark = pytest.mark.gpu


def oracle_star(fact, dims):
    s1 = oracle.select(dims["d1_c5"], oracle.EQ, 0)
    s2 = oracle.select(dims["d2_c25"], oracle.LT, 15)
    p1 = oracle.semijoin(fact["fk1"], s1, synth.DIM_SIZES[0])
    q2 = oracle.semijoin(oracle.project(fact["fk2"], p1), s2, synth.DIM_SIZES[1])
    p2 = oracle.project(p1, q2)
    p3 = oracle.project(p2, oracle.select(oracle.project(fact["discount"], p2), oracle.BETWEEN, 1, 3))
    p4 = oracle.project(p3, oracle.select(oracle.project(fact["quantity"], p3), oracle.LT, 25))
    year = oracle.project(dims["date_year"], oracle.project(fact["fk_date"], p4))
    c25 = oracle.project(dims["d2_c25"], oracle.project(fact["fk2"], p4))
    gid = oracle.calc(oracle.ADD, oracle.calc(oracle.MUL, year, c=15), c25)
    return oracle.group_sum(gid, oracle.project(fact["revenue"], p4), plans.STAR_GROUPS), p4.size


@pytest.mark.parametrize("base_fm,fm", [(plans.STAR_BASE_COMPRESSED, plans.STAR_COMPRESSED),
                                        (plans.STAR_BASE_UNCOMPRESSED, plans.STAR_UNCOMPRESSED),
                                        (plans.STAR_BASE_COMPRESSED, plans.STAR_UNCOMPRESSED)])
def test_star_plan_matches_oracle(base_fm, fm):
    n = (1 << 20) + 333
    fact = synth.star_fact(3, n)
    dims = synth.star_dims(4)
    want, matched = oracle_star(fact, dims)
    assert 0.01 < matched / n < 0.022  # 0.2 * 0.6 * 3/11 * 24/50 = 1.57%
    with ms.Ctx(0, arena_bytes=1 << 30, max_rows=1 << 22) as ctx:
        base = plans.compress_base(ctx, {k: ms.as_device_u64(v, ctx.device) for k, v in {**fact, **dims}.items()},
                                   base_fm)
        res, cols = plans.star_plan(ctx, base, fm)
        got = ms.to_numpy_u64(res)
        ctx.check(what="star plan")
        np.testing.assert_array_equal(got, want)
        assert plans.footprint(ctx, cols) > 0
        plans.free_lifo(ctx, cols)


@pytest.mark.parametrize("base_fm,fm", [(plans.STAR_BASE_COMPRESSED, plans.STAR_COMPRESSED),
                                        (plans.STAR_BASE_UNCOMPRESSED, plans.STAR_UNCOMPRESSED)])
def test_star_plan_intermediates_match_oracle(base_fm, fm):
    """Every intermediate of the star plan against the oracle's, checked right
    after its operator (the first divergent operator names itself)."""
    n = (1 << 18) + 77
    fact = synth.star_fact(5, n)
    dims = synth.star_dims(6)
    D = synth.DIM_SIZES
    with ms.Ctx(0, arena_bytes=1 << 30, max_rows=1 << 20) as ctx:
        base = plans.compress_base(ctx, {k: ms.as_device_u64(v, ctx.device) for k, v in {**fact, **dims}.items()},
                                   base_fm)
        assert ctx.get_error() == ms.MS_OK
        want, got = {}, {}
        steps = [
            ("S1", lambda: oracle.select(dims["d1_c5"], oracle.EQ, 0),
             lambda: ctx.select(base["d1_c5"], ms.EQ, 0, fmt=fm["S1"])),
            ("S2", lambda: oracle.select(dims["d2_c25"], oracle.LT, 15),
             lambda: ctx.select(base["d2_c25"], ms.LT, 15, fmt=fm["S2"])),
            ("P1", lambda: oracle.semijoin(fact["fk1"], want["S1"], D[0]),
             lambda: ctx.semijoin(base["fk1"], got["S1"], D[0], fmt=fm["P1"])),
            ("F2", lambda: oracle.project(fact["fk2"], want["P1"]),
             lambda: ctx.project(base["fk2"], got["P1"], fmt=fm["F2"], bw=plans.star_width("F2", fm["F2"]))),
            ("Q2", lambda: oracle.semijoin(want["F2"], want["S2"], D[1]),
             lambda: ctx.semijoin(got["F2"], got["S2"], D[1], fmt=fm["Q2"])),
            ("P2", lambda: oracle.project(want["P1"], want["Q2"]),
             lambda: ctx.project(got["P1"], got["Q2"], fmt=fm["P2"])),
            ("DISC", lambda: oracle.project(fact["discount"], want["P2"]),
             lambda: ctx.project(base["discount"], got["P2"], fmt=fm["DISC"], bw=plans.star_width("DISC", fm["DISC"]))),
            ("Q3", lambda: oracle.select(want["DISC"], oracle.BETWEEN, 1, 3),
             lambda: ctx.select(got["DISC"], ms.BETWEEN, 1, 3, fmt=fm["Q3"])),
            ("P3", lambda: oracle.project(want["P2"], want["Q3"]),
             lambda: ctx.project(got["P2"], got["Q3"], fmt=fm["P3"])),
            ("QTY", lambda: oracle.project(fact["quantity"], want["P3"]),
             lambda: ctx.project(base["quantity"], got["P3"], fmt=fm["QTY"], bw=plans.star_width("QTY", fm["QTY"]))),
            ("Q4", lambda: oracle.select(want["QTY"], oracle.LT, 25),
             lambda: ctx.select(got["QTY"], ms.LT, 25, fmt=fm["Q4"])),
            ("P4", lambda: oracle.project(want["P3"], want["Q4"]),
             lambda: ctx.project(got["P3"], got["Q4"], fmt=fm["P4"])),
            ("DATE", lambda: oracle.project(fact["fk_date"], want["P4"]),
             lambda: ctx.project(base["fk_date"], got["P4"], fmt=fm["DATE"])),
            ("YEAR", lambda: oracle.project(dims["date_year"], want["DATE"]),
             lambda: ctx.project(base["date_year"], got["DATE"], fmt=fm["YEAR"], bw=plans.star_width("YEAR", fm["YEAR"]))),
            ("F2B", lambda: oracle.project(fact["fk2"], want["P4"]),
             lambda: ctx.project(base["fk2"], got["P4"], fmt=fm["F2B"], bw=plans.star_width("F2B", fm["F2B"]))),
            ("C25", lambda: oracle.project(dims["d2_c25"], want["F2B"]),
             lambda: ctx.project(base["d2_c25"], got["F2B"], fmt=fm["C25"], bw=plans.star_width("C25", fm["C25"]))),
            ("G0", lambda: oracle.calc(oracle.MUL, want["YEAR"], c=15),
             lambda: ctx.calc(ms.MUL, got["YEAR"], None, c=15, fmt=fm["G0"], bw=plans.star_width("G0", fm["G0"]))),
            ("GID", lambda: oracle.calc(oracle.ADD, want["G0"], want["C25"]),
             lambda: ctx.calc(ms.ADD, got["G0"], got["C25"], fmt=fm["GID"], bw=plans.star_width("GID", fm["GID"]))),
            ("REV", lambda: oracle.project(fact["revenue"], want["P4"]),
             lambda: ctx.project(base["revenue"], got["P4"], fmt=fm["REV"], bw=plans.star_width("REV", fm["REV"]))),
        ]
        for name, w, g in steps:
            want[name] = w()
            got[name] = g()
            code = ctx.get_error()
            assert code == ms.MS_OK, f"device error {code} (info {ctx.last_error_info()}) by {name}"
            np.testing.assert_array_equal(ms.to_numpy_u64(ctx.decompress(got[name])), want[name], err_msg=name)


@pytest.mark.parametrize("objective", ["size", "time"])
def test_greedy_plan_formats_keep_results_and_meet_their_objective(objective):
    """Plan-level format choice (Sec. 5.2): the greedy per-intermediate search over the
    star plan's 19 intermediates changes formats only (the sums stay the oracle's),
    and its combination costs no more than the starting one under its objective."""
    n = (1 << 18) + 5
    fact = synth.star_fact(9, n)
    dims = synth.star_dims(10)
    want, _ = oracle_star(fact, dims)
    with ms.Ctx(0, arena_bytes=1 << 30, max_rows=1 << 20) as ctx:
        base = plans.compress_base(ctx, {k: ms.as_device_u64(v, ctx.device) for k, v in {**fact, **dims}.items()},
                                   plans.STAR_BASE_COMPRESSED)
        run = lambda fm: plans.star_plan(ctx, base, fm)  # noqa: E731
        start = dict(plans.STAR_COMPRESSED)
        c0 = plans.plan_cost(ctx, run, start, objective, reps=2)
        fm, c, evals = plans.greedy_formats(ctx, run, plans.STAR_NAMES, start, objective,
                                            candidates=plans.STAR_CANDIDATES, reps=2)
        assert evals == sum(len(plans.STAR_CANDIDATES[name]) for name in plans.STAR_NAMES)
        if objective == "size":  # sizes are deterministic: the search can only improve
            assert c <= c0 and plans.plan_cost(ctx, run, fm, "size") == c
        res, cols = run(fm)
        ctx.check(what="greedy formats")
        np.testing.assert_array_equal(ms.to_numpy_u64(res), want)
        plans.free_lifo(ctx, cols)
