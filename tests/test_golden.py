"""Pins of the measurement model to values the paper prints.

The paper's only worked example (Sec. III-B, an 8n x n matrix in four row
blocks) is structural and is checked in the oracle tests; its printed numbers
are the per-step byte counts of the performance model (Sec. V-A table), stored
in tests/golden/reads_writes_per_step.txt.  The algorithmic bytes per row that
bench.py reports (in units of n s, s = bytes per element) must equal the
paper's tall-matrix value bytes (the terms in m n) for each method.
"""
import os
from collections import defaultdict

import bench

HERE = os.path.dirname(os.path.abspath(__file__))


def _table():
    t = defaultdict(dict)
    with open(os.path.join(HERE, "golden", "reads_writes_per_step.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            method, step, c_mn, c_m1n2 = line.split()
            t[method][step] = (int(c_mn), int(c_m1n2))
    return t


def test_tall_bytes_match_the_paper():
    t = _table()
    tall = {meth: sum(c for c, _ in steps.values()) for meth, steps in t.items()}
    # the paper counts doubles: 8 m n bytes per pass over the tall matrix
    assert tall["direct"] == 8 * bench.ALG_PASSES["direct"]
    assert tall["cholesky"] == 8 * bench.ALG_PASSES["cholqr"]
    assert tall["indirect"] == 8 * bench.ALG_PASSES["indirect"]
    # one refinement step repeats the method on the computed Q (Sec. I)
    assert bench.ALG_PASSES["cholqr_ir"] == 2 * bench.ALG_PASSES["cholqr"]
    assert bench.ALG_PASSES["indirect_ir"] == 2 * bench.ALG_PASSES["indirect"]


def test_direct_stack_bytes_are_small():
    """The stacked R factors (terms in m1 n^2) are the only non-tall traffic of
    direct TSQR: per block one n x n R written in step 1 and read in step 2."""
    t = _table()
    assert t["direct"]["W1m"][1] == 8 and t["direct"]["R2m"][1] == 8
