"""Randomized checks of the task-list builder over shapes, tile sizes, modes
and variants (flat, reduction tree, 2b x b bottoms, tiled LU, explicit Q):
every list the library would launch must be accepted by its own rule check
(each writer waits for exactly the writers before it in the sequential
order), be a topological order of the waits, and hold each task once."""
import numpy as np
import pytest

from paper_0707_3548_gb300 import tqr
from tests.test_plan import Grid, check_order_satisfies_waits

FACTOR, APPLY_QT, APPLY_Q, TRSM, TRSMT, FORM_Q = range(6)
LUF, PAIR = 16, 32


def _cases(seed, count):
    g = np.random.default_rng(seed)
    out = []
    while len(out) < count:
        nb = int(g.choice([8, 16, 24]))       # the library takes nb multiple of 8 in [8, 256]
        ib = int(g.choice([x for x in (1, 2, 4, 8, 16) if x <= nb and nb % x == 0]))
        cs = int(g.choice([x for x in (1, 2, 4, 8) if x <= nb and nb % x == 0]))
        m = int(g.integers(1, 9 * nb))
        n = int(g.integers(1, 6 * nb))
        nrhs = int(g.integers(1, 3 * nb))
        variant = str(g.choice(["flat", "tree", "pair", "lu", "lupair"]))
        mode = int(g.choice([FACTOR, APPLY_QT, APPLY_Q, TRSM, TRSMT, FORM_Q]))
        D = int(g.integers(1, 5)) if variant == "tree" else 0
        if variant in ("lu", "lupair") and mode not in (FACTOR, APPLY_QT, TRSM):
            continue
        if mode == FORM_Q and variant not in ("flat", "tree"):
            continue
        trsm = int(g.integers(0, 2)) if mode in (FACTOR, APPLY_QT) and m >= n else 0
        if mode == FACTOR and not trsm:
            nrhs = int(g.integers(0, 2)) * nrhs
        flag = {"flat": 0, "tree": 0, "pair": PAIR, "lu": LUF, "lupair": LUF | PAIR}[variant]
        out.append((m, n, nb, ib, cs, nrhs, mode | flag, trsm, D))
    return out


@pytest.mark.parametrize("case", _cases(7, 400))
def test_random_plans_are_valid_orders(case):
    m, n, nb, ib, cs, nrhs, mode, trsm, D = case
    tasks, stats = tqr.tqr_debug_plan(mode, m, n, nb, ib, cs, nrhs, trsm, 5, -1, D=D)
    keys = [tuple(int(v) for v in t[:7]) for t in tasks]
    assert len(set(keys)) == len(keys)
    g = Grid(m, n, nb, ib, cs, nrhs)
    # rules with the same mode flags and D as the plan
    ver = {}
    for t in tasks:
        waits, sigs = tqr.tqr_debug_rules(mode, m, n, nb, ib, cs, nrhs, t[:7], D=D)
        for ctr, cnt, v in waits:
            for c in range(cnt):
                assert ver.get(ctr + c, 0) >= v, (case, t, ctr + c, v)
        for ctr, cnt in sigs:
            for c in range(cnt):
                ver[ctr + c] = ver.get(ctr + c, 0) + 1
    if len(tasks):
        assert stats[4] <= stats[0] * (1 + 1e-9)          # critical path <= simulated makespan
    lean, _ = tqr.tqr_debug_plan(mode, m, n, nb, ib, cs, nrhs, trsm, 5, 2, D=D)
    assert sorted(tuple(int(v) for v in t[:7]) for t in lean) == sorted(keys)
