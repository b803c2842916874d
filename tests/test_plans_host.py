"""Host logic of the plan-level format search (Sec. 5.2, greedy per-intermediate
choice), with an injected cost function: no GPU."""
import itertools

import pytest

from paper_2004_09350_gb300 import morphstore as ms
from paper_2004_09350_gb300 import plans


def _additive_cost(table):
    # cost of a combination = sum of per-intermediate costs: the greedy search is
    # then exact, and equals the brute-force minimum
    return lambda fm: sum(table[name][fmt] for name, fmt in fm.items())


def test_greedy_is_exact_for_separable_costs():
    names = ["A", "B", "C"]
    table = {"A": {ms.UNCOMPR: 5, ms.DYN_BP: 1, ms.DELTA_BP: 3, ms.FOR_BP: 2},
             "B": {ms.UNCOMPR: 2, ms.DYN_BP: 4, ms.DELTA_BP: 0.5, ms.FOR_BP: 9},
             "C": {ms.UNCOMPR: 1, ms.DYN_BP: 1.5, ms.DELTA_BP: 7, ms.FOR_BP: 0.25}}
    fm, c, evals = plans.greedy_formats(None, None, names, {n: ms.UNCOMPR for n in names},
                                        cost=_additive_cost(table))
    assert fm == {"A": ms.DYN_BP, "B": ms.DELTA_BP, "C": ms.FOR_BP}
    brute = min(itertools.product(plans.PLAN_CANDIDATES, repeat=3),
                key=lambda f: _additive_cost(table)(dict(zip(names, f))))
    assert tuple(fm[n] for n in names) == brute
    assert c == pytest.approx(1 + 0.5 + 0.25)
    assert evals == 3 * len(plans.PLAN_CANDIDATES)


def test_greedy_visits_in_plan_order_and_keeps_earlier_choices():
    # an interaction term: B's best format depends on A's; the search fixes A first
    seen = []

    def cost(fm):
        seen.append(dict(fm))
        base = {ms.UNCOMPR: 4, ms.DYN_BP: 1, ms.DELTA_BP: 2, ms.FOR_BP: 3}[fm["A"]]
        inter = 0 if fm["B"] == fm["A"] else 2
        return base + inter

    fm, c, _ = plans.greedy_formats(None, None, ["A", "B"], {"A": ms.UNCOMPR, "B": ms.UNCOMPR}, cost=cost)
    assert fm == {"A": ms.DYN_BP, "B": ms.DYN_BP} and c == 1
    k = len(plans.PLAN_CANDIDATES)
    assert all(s["B"] == ms.UNCOMPR for s in seen[:k])   # A first, B held at its start
    assert all(s["A"] == ms.DYN_BP for s in seen[k:])    # then B, with A fixed


def test_greedy_rejects_unknown_objective():
    with pytest.raises(ValueError):
        plans.greedy_formats(None, None, ["A"], {"A": 0}, objective="energy", cost=lambda fm: 0)


def test_star_plan_tables_cover_every_intermediate():
    assert set(plans.STAR_NAMES) == set(plans.STAR_COMPRESSED) == set(plans.STAR_OPS)
    assert set(plans.STAR_RANDOM_READS) <= set(plans.STAR_NAMES)
