"""Operator-at-a-time query plans over the C ABI (paper Sec. 3.3: every operator
runs to completion and materialises its output column in its own format).

Each plan takes a ``morphstore.Ctx``, base columns and a map from intermediate name
to format, enqueues its operators on the current stream without host syncs, and
returns its result tensor plus the intermediates (newest last), so the caller can
read their sizes (the paper's footprint, Sec. 5.2) and free them LIFO.
"""
from __future__ import annotations

from . import morphstore as ms

# ------------------------------------------------------------- simple plans


def select_project_sum(ctx, x, y, c, fm, out=None):
    """SUM(Y) WHERE X < c (Sec. 5.1 "Simple Query" with a range predicate)."""
    pos = ctx.select(x, ms.LT, c, fmt=fm["P"])
    yp = ctx.project(y, pos, fmt=fm["Y'"])
    res = ctx.agg_sum(yp, out=out)
    return res, [pos, yp]


def select_project_calc_sum(ctx, x, k, c, fm, out=None):
    """select(X < c) -> P; project X and K at P; calc X' * K'; sum."""
    pos = ctx.select(x, ms.LT, c, fmt=fm["P"])
    xp = ctx.project(x, pos, fmt=fm["X'"])
    kp = ctx.project(k, pos, fmt=fm["K'"])
    y = ctx.calc(ms.MUL, xp, kp, fmt=fm["Y"])
    res = ctx.agg_sum(y, out=out)
    return res, [pos, xp, kp, y]


# ------------------------------------------------------------ star schema

STAR_GROUPS = 105  # year (7 values) * 15 + c25 (< 15 after the filter)

STAR_COMPRESSED = {
    # positions are sorted: DELTA+BP (so are the projected dates); values: static BP at the
    # width of their value domain (STAR_VALUE_WIDTHS), which needs no placement pass
    "S1": ms.DELTA_BP, "S2": ms.DELTA_BP, "P1": ms.DELTA_BP, "F2": ms.STATIC_BP, "Q2": ms.DELTA_BP,
    "P2": ms.DELTA_BP, "DISC": ms.STATIC_BP, "Q3": ms.DELTA_BP, "P3": ms.DELTA_BP, "QTY": ms.STATIC_BP,
    "Q4": ms.DELTA_BP, "P4": ms.DELTA_BP, "DATE": ms.DELTA_BP, "YEAR": ms.STATIC_BP, "F2B": ms.STATIC_BP,
    "C25": ms.STATIC_BP, "G0": ms.STATIC_BP, "GID": ms.STATIC_BP, "REV": ms.STATIC_BP,
}
STAR_UNCOMPRESSED = {k: ms.UNCOMPR for k in STAR_COMPRESSED}
# Value intermediates whose domain the plan knows before they exist: fk2 < 2e5 (F2, F2B),
# discount <= 10, quantity <= 50, year < 7, c25 < 25, year * 15 <= 90, year * 15 + c25
# < 105, revenue < 2^23.  Static BP at these widths is a candidate for them; a value
# beyond its width raises MS_ERR_VALUE_TOO_WIDE.
STAR_VALUE_WIDTHS = {"F2": 18, "DISC": 4, "QTY": 6, "YEAR": 3, "F2B": 18, "C25": 5, "G0": 7, "GID": 7,
                     "REV": 23}


def star_width(name: str, fmt: int) -> int:
    """Static-BP width of star intermediate `name` in format fmt (0 for other formats)."""
    return STAR_VALUE_WIDTHS[name] if fmt == ms.STATIC_BP else 0

# Base columns.  Sec. 4.2 allows random access only into uncompressed and static-BP
# columns: the columns that the plan projects at positions (fk2, discount, quantity,
# revenue, d2_c25, date_year) are static BP at the width of their value domain, so a
# value is read without a block header; the sorted date key is DELTA+BP; the columns
# that are only scanned are dynamic BP.
STAR_BASE_COMPRESSED = {"fk1": ms.DYN_BP, "fk2": ms.STATIC_BP, "fk3": ms.DYN_BP, "fk_date": ms.DELTA_BP,
                        "quantity": ms.STATIC_BP, "discount": ms.STATIC_BP, "revenue": ms.STATIC_BP,
                        "d1_c5": ms.DYN_BP, "d2_c25": ms.STATIC_BP, "date_year": ms.STATIC_BP}
STAR_BASE_UNCOMPRESSED = {k: ms.UNCOMPR for k in STAR_BASE_COMPRESSED}
# static-BP widths: the value domains of the generated columns (fk2 < 2e5, quantity
# <= 50, discount <= 10, revenue < 2^23, c25 < 25, year < 7)
STAR_BASE_WIDTHS = {"fk2": 18, "quantity": 6, "discount": 4, "revenue": 23, "d2_c25": 5, "date_year": 3}


def base_width(name: str, fmt: int) -> int:
    """Static-BP width of a star base column in format fmt (0 for other formats)."""
    return STAR_BASE_WIDTHS[name] if fmt == ms.STATIC_BP else 0


def compress_base(ctx, cols, formats):
    """The star plan's base columns (device tensors by name) compressed in `formats`."""
    return {k: ctx.compress(v, formats[k], base_width(k, formats[k])) for k, v in cols.items()}


def star_plan(ctx, base, fm, out=None, trace=None):
    """Star-schema plan: select on two dimensions, semi-join them into the fact
    table, select on discount and quantity ranges, project, and group-sum revenue
    by (year, c25):

      S1 = sigma(D1.c5 = 0); S2 = sigma(D2.c25 < 15)
      P1 = fact rows with fk1 in S1; P2 = P1 rows with fk2 in S2
      P3 = P2 rows with 1 <= discount <= 3; P4 = P3 rows with quantity < 25
      gid = year(fk_date) * 15 + D2.c25[fk2]; result[g] = sum of revenue per gid

    trace, when a list, receives one record per operator: (op, output name,
    input columns, output column, key domain or group count, CUDA events before
    and after the operator's launches).
    """
    from .synth import DIM_SIZES
    cols = []
    ev = [None]

    def mark():  # an event before the next operator's launches (traced runs only)
        if trace is not None:
            import torch
            ev[0] = torch.cuda.Event(enable_timing=True)
            ev[0].record()

    def keep(op, name, ins, c, extra=0):
        cols.append(c)
        if trace is not None:
            import torch
            e1 = torch.cuda.Event(enable_timing=True)
            e1.record()
            trace.append((op, name, ins, c, extra, ev[0], e1))
        mark()
        return c

    mark()

    b = base
    s1 = keep("select", "S1", [b["d1_c5"]], ctx.select(b["d1_c5"], ms.EQ, 0, fmt=fm["S1"]))
    s2 = keep("select", "S2", [b["d2_c25"]], ctx.select(b["d2_c25"], ms.LT, 15, fmt=fm["S2"]))
    p1 = keep("semijoin", "P1", [b["fk1"], s1], ctx.semijoin(b["fk1"], s1, DIM_SIZES[0], fmt=fm["P1"]), DIM_SIZES[0])
    f2 = keep("project", "F2", [b["fk2"], p1], ctx.project(b["fk2"], p1, fmt=fm["F2"], bw=star_width("F2", fm["F2"])))
    q2 = keep("semijoin", "Q2", [f2, s2], ctx.semijoin(f2, s2, DIM_SIZES[1], fmt=fm["Q2"]), DIM_SIZES[1])
    p2 = keep("project", "P2", [p1, q2], ctx.project(p1, q2, fmt=fm["P2"]))
    disc = keep("project", "DISC", [b["discount"], p2], ctx.project(b["discount"], p2, fmt=fm["DISC"], bw=star_width("DISC", fm["DISC"])))
    q3 = keep("select", "Q3", [disc], ctx.select(disc, ms.BETWEEN, 1, 3, fmt=fm["Q3"]))
    p3 = keep("project", "P3", [p2, q3], ctx.project(p2, q3, fmt=fm["P3"]))
    qty = keep("project", "QTY", [b["quantity"], p3], ctx.project(b["quantity"], p3, fmt=fm["QTY"], bw=star_width("QTY", fm["QTY"])))
    q4 = keep("select", "Q4", [qty], ctx.select(qty, ms.LT, 25, fmt=fm["Q4"]))
    p4 = keep("project", "P4", [p3, q4], ctx.project(p3, q4, fmt=fm["P4"]))
    date = keep("project", "DATE", [b["fk_date"], p4], ctx.project(b["fk_date"], p4, fmt=fm["DATE"]))
    year = keep("project", "YEAR", [b["date_year"], date], ctx.project(b["date_year"], date, fmt=fm["YEAR"], bw=star_width("YEAR", fm["YEAR"])))
    f2b = keep("project", "F2B", [b["fk2"], p4], ctx.project(b["fk2"], p4, fmt=fm["F2B"], bw=star_width("F2B", fm["F2B"])))
    c25 = keep("project", "C25", [b["d2_c25"], f2b], ctx.project(b["d2_c25"], f2b, fmt=fm["C25"], bw=star_width("C25", fm["C25"])))
    g0 = keep("calc", "G0", [year], ctx.calc(ms.MUL, year, None, c=15, fmt=fm["G0"], bw=star_width("G0", fm["G0"])))
    gid = keep("calc", "GID", [g0, c25], ctx.calc(ms.ADD, g0, c25, fmt=fm["GID"], bw=star_width("GID", fm["GID"])))
    rev = keep("project", "REV", [b["revenue"], p4], ctx.project(b["revenue"], p4, fmt=fm["REV"], bw=star_width("REV", fm["REV"])))
    res = ctx.group_sum(gid, rev, STAR_GROUPS, out=out)
    if trace is not None:
        import torch
        e1 = torch.cuda.Event(enable_timing=True)
        e1.record()
        trace.append(("group_sum", "RESULT", [gid, rev], None, STAR_GROUPS, ev[0], e1))
    return res, cols


def free_lifo(ctx, cols):
    for c in reversed(cols):
        ctx.free(c)


def footprint(ctx, cols) -> int:
    """Sum of the physical sizes of the given columns (synchronises)."""
    return sum(ctx.info(c)["size_bytes"] for c in cols)


# --------------------------------------------- plan-level format choice

# Formats an intermediate may take when the choice is made before it exists: static
# BP needs its width up front, so it is left to the selector's sampled statistics.
PLAN_CANDIDATES = (ms.UNCOMPR, ms.DYN_BP, ms.DELTA_BP, ms.FOR_BP)
PLAN_OBJECTIVES = ("time", "size")


def plan_cost(ctx, run, fm, objective="time", reps=3):
    """Cost of one format combination of a plan.  run(fm) enqueues the plan and
    returns (result, intermediates in allocation order).  objective "time": mean
    device milliseconds of `reps` runs after one warm-up run (CUDA events on the
    current stream); "size": the sum of the intermediates' physical sizes (the
    paper's footprint measure, Sec. 5.2).  Every run frees its intermediates."""
    import torch
    _, cols = run(fm)
    if objective == "size":
        cost = footprint(ctx, cols)
        free_lifo(ctx, cols)
        return float(cost)
    free_lifo(ctx, cols)
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(reps):
        _, cols = run(fm)
        free_lifo(ctx, cols)
    t1.record()
    t1.synchronize()
    return t0.elapsed_time(t1) / reps


def greedy_formats(ctx, run, names, start, objective="time", candidates=PLAN_CANDIDATES, reps=3, cost=None):
    """Greedy per-intermediate format search over a whole plan (Sec. 5.2,
    "Determining a good format combination"): the intermediates are visited once,
    in plan order; for each, every candidate format is tried with all others held
    fixed, and the cheapest is kept before moving on.  Returns (formats, cost of
    the final combination, number of plan evaluations).  `candidates` is one tuple
    for every intermediate or a dict of tuples by name; `cost(fm)` overrides the
    measurement (plan_cost by default)."""
    if objective not in PLAN_OBJECTIVES:
        raise ValueError(f"objective must be one of {PLAN_OBJECTIVES}")
    measure = cost or (lambda fm: plan_cost(ctx, run, fm, objective, reps))
    fm = dict(start)
    evals, best_cost = 0, None
    for name in names:
        best = None
        for f in (candidates[name] if isinstance(candidates, dict) else candidates):
            trial = dict(fm, **{name: f})
            c = measure(trial)
            evals += 1
            if best is None or c < best[0]:
                best = (c, f)
        fm[name] = best[1]
        best_cost = best[0]
    return fm, best_cost, evals


def selector_formats(ctx, selector, run_sample, names, ops, objective="time", candidates=PLAN_CANDIDATES,
                     n_scale=1.0, random_reads=()):
    """Formats chosen by the learned selector (selector.Selector) before the plan
    runs: run_sample(fm) runs the plan once on a prefix sample with every
    intermediate uncompressed; each intermediate's statistics (ms_column_stats),
    scaled to the full length by n_scale, give its features, and the selector picks
    the format it predicts cheapest for the objective.  ops[name] is the producing
    operator ("select", "project", "calc", "semijoin"); names in random_reads are
    read at random by a later project."""
    from . import selector as sel_mod
    fm0 = {name: ms.UNCOMPR for name in names}
    _, cols = run_sample(fm0)
    feats = []
    for name, col in zip(names, cols):
        feats.append(sel_mod.column_features(ctx, col, ops[name], name in random_reads, n_scale))
    free_lifo(ctx, cols)
    picks = selector.choose(__import__("numpy").stack(feats), objective, allowed=candidates)
    return {name: int(p) for name, p in zip(names, picks)}


STAR_NAMES = tuple(STAR_COMPRESSED)  # the star plan's intermediates in plan order
STAR_OPS = {"S1": "select", "S2": "select", "P1": "semijoin", "F2": "project", "Q2": "semijoin", "P2": "project",
            "DISC": "project", "Q3": "select", "P3": "project", "QTY": "project", "Q4": "select", "P4": "project",
            "DATE": "project", "YEAR": "project", "F2B": "project", "C25": "project", "G0": "calc", "GID": "calc",
            "REV": "project"}
# intermediates a later project reads at random (the position lists projected through)
STAR_RANDOM_READS = ("P1", "P2", "P3")
# greedy-search candidates of the star plan: static BP too where the value width is known
STAR_CANDIDATES = {name: PLAN_CANDIDATES + ((ms.STATIC_BP,) if name in STAR_VALUE_WIDTHS else ())
                   for name in STAR_NAMES}
