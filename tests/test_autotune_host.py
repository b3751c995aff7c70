"""The autotuner's search space and the committed tuning table, on the host:
every candidate entry is one the planner accepts, the committed table loads
and is valid, and a plan made with it covers a mixed batch."""
import json
import os

import numpy as np

import paper_2108_02025_gb300 as gb
from paper_2108_02025_gb300 import autotune
from test_batch_plan import FakeBatch


def plan_ok(table):
    one = np.array([100], np.int64)
    return gb.gb_sgemv_batch_plan_bytes(1, one, one, np.array([1.0], np.float32), table) > 0


def test_every_candidate_is_a_valid_entry():
    for b in range(5, 14):
        cands = list(autotune.candidates(b))
        assert cands, b
        for lpr, u, tb in cands:
            assert plan_ok(gb.tuning_table({b: (lpr, u, tb)})), (b, lpr, u, tb)
        # no candidate spreads a row over more lanes than twice its packs
        packs = max(1, (1 << b) // 4)
        assert all(lpr <= max(1, 2 * packs) for lpr, _, _ in cands)


def test_committed_table_loads_and_plans():
    path = gb.TUNING_PATH
    assert os.path.exists(path)
    with open(path) as f:
        json.load(f)
    table = gb.load_tuning()
    assert plan_ok(table)
    fb = FakeBatch([5, 100, 3000, 40], [4000, 33, 700, 8192])
    st, _ = fb.plan(table)
    assert st == gb.GB_OK
