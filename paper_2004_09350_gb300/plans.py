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
    # positions are sorted: DELTA+BP; values: dynamic BP
    "S1": ms.DELTA_BP, "S2": ms.DELTA_BP, "P1": ms.DELTA_BP, "F2": ms.DYN_BP, "Q2": ms.DELTA_BP,
    "P2": ms.DELTA_BP, "DISC": ms.DYN_BP, "Q3": ms.DELTA_BP, "P3": ms.DELTA_BP, "QTY": ms.DYN_BP,
    "Q4": ms.DELTA_BP, "P4": ms.DELTA_BP, "DATE": ms.DELTA_BP, "YEAR": ms.DYN_BP, "F2B": ms.DYN_BP,
    "C25": ms.DYN_BP, "G0": ms.DYN_BP, "GID": ms.DYN_BP, "REV": ms.DYN_BP,
}
STAR_UNCOMPRESSED = {k: ms.UNCOMPR for k in STAR_COMPRESSED}

STAR_BASE_COMPRESSED = {"fk1": ms.DYN_BP, "fk2": ms.DYN_BP, "fk3": ms.DYN_BP, "fk_date": ms.DELTA_BP,
                        "quantity": ms.DYN_BP, "discount": ms.DYN_BP, "revenue": ms.DYN_BP,
                        "d1_c5": ms.DYN_BP, "d2_c25": ms.DYN_BP, "date_year": ms.DYN_BP}
STAR_BASE_UNCOMPRESSED = {k: ms.UNCOMPR for k in STAR_BASE_COMPRESSED}


def star_plan(ctx, base, fm, out=None):
    """Star-schema plan: select on two dimensions, semi-join them into the fact
    table, select on discount and quantity ranges, project, and group-sum revenue
    by (year, c25):

      S1 = sigma(D1.c5 = 0); S2 = sigma(D2.c25 < 15)
      P1 = fact rows with fk1 in S1; P2 = P1 rows with fk2 in S2
      P3 = P2 rows with 1 <= discount <= 3; P4 = P3 rows with quantity < 25
      gid = year(fk_date) * 15 + D2.c25[fk2]; result[g] = sum of revenue per gid
    """
    from .synth import DIM_SIZES
    cols = []

    def keep(c):
        cols.append(c)
        return c

    s1 = keep(ctx.select(base["d1_c5"], ms.EQ, 0, fmt=fm["S1"]))
    s2 = keep(ctx.select(base["d2_c25"], ms.LT, 15, fmt=fm["S2"]))
    p1 = keep(ctx.semijoin(base["fk1"], s1, DIM_SIZES[0], fmt=fm["P1"]))
    f2 = keep(ctx.project(base["fk2"], p1, fmt=fm["F2"]))
    q2 = keep(ctx.semijoin(f2, s2, DIM_SIZES[1], fmt=fm["Q2"]))
    p2 = keep(ctx.project(p1, q2, fmt=fm["P2"]))
    disc = keep(ctx.project(base["discount"], p2, fmt=fm["DISC"]))
    q3 = keep(ctx.select(disc, ms.BETWEEN, 1, 3, fmt=fm["Q3"]))
    p3 = keep(ctx.project(p2, q3, fmt=fm["P3"]))
    qty = keep(ctx.project(base["quantity"], p3, fmt=fm["QTY"]))
    q4 = keep(ctx.select(qty, ms.LT, 25, fmt=fm["Q4"]))
    p4 = keep(ctx.project(p3, q4, fmt=fm["P4"]))
    date = keep(ctx.project(base["fk_date"], p4, fmt=fm["DATE"]))
    year = keep(ctx.project(base["date_year"], date, fmt=fm["YEAR"]))
    f2b = keep(ctx.project(base["fk2"], p4, fmt=fm["F2B"]))
    c25 = keep(ctx.project(base["d2_c25"], f2b, fmt=fm["C25"]))
    g0 = keep(ctx.calc(ms.MUL, year, None, c=15, fmt=fm["G0"]))
    gid = keep(ctx.calc(ms.ADD, g0, c25, fmt=fm["GID"]))
    rev = keep(ctx.project(base["revenue"], p4, fmt=fm["REV"]))
    res = ctx.group_sum(gid, rev, STAR_GROUPS, out=out)
    return res, cols


def free_lifo(ctx, cols):
    for c in reversed(cols):
        ctx.free(c)


def footprint(ctx, cols) -> int:
    """Sum of the physical sizes of the given columns (synchronises)."""
    return sum(ctx.info(c)["size_bytes"] for c in cols)
