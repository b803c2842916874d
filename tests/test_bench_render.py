"""Host-side checks of bench.py helpers: the committed sweep-table markdown is the
rendering of the committed sweep-table line, and the static cascade width the sweep
uses is the widest block's residual width as the oracle computes it."""
import json
import os

import numpy as np
import pytest

import bench
import oracle
from paper_2004_09350_gb300 import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_committed_sweep_table_markdown_is_its_json_rendered():
    with open(os.path.join(ROOT, "profiles", "sweep_table_2e28.json")) as f:
        line = json.loads(f.read().strip().splitlines()[-1])
    with open(os.path.join(ROOT, "profiles", "sweep_table_2e28.md")) as f:
        md = f.read()
    assert bench.render_sweep_table(line).strip() == md.strip()


@pytest.mark.parametrize("n", [100, 512, 5000, 3 * 512 + 7])
def test_cascade_width_matches_the_oracle(n):
    k = synth.sorted_gaps(5, n)
    x = synth.skewed_widths(6, n)
    want_k = int(oracle.block_widths(oracle.DELTA_BP, k).max()) if n >= 512 else 1
    want_x = int(oracle.block_widths(oracle.FOR_BP, x).max()) if n >= 512 else 1
    assert max(1, bench.oracle_free_block_width(k, True)) == max(1, want_k)
    assert max(1, bench.oracle_free_block_width(x, False)) == max(1, want_x)
