"""Host logic of the tiled LU's task lists, checked on the CPU: the plans the
library would launch (tqr_debug_plan with the LU flag) are replayed slab by
slab with the oracle's LU tile kernels, in plan order and in random orders
that respect the version waits, and must reproduce the oracle's sequential
factorization and solve."""
import numpy as np
import pytest

from oracle import tiled_lu as LU
from paper_0707_3548_gb300 import inputs, tqr
from tests.test_plan import APPLY_QT, FACTOR, Grid, check_order_satisfies_waits, random_valid_order

LUF = 16
TRSM_UPD, TRSM_SOLVE = 6, 7
GETRF, GESSM, TSTRF, SSSSM = 13, 14, 15, 16


class LuGrid(Grid):
    def __init__(self, *a, **k):
        super().__init__(*a, **k)
        self.piv = {}
        self.L1 = {}


def execute(g, task):
    kind, s, _, k, i, j, l = (int(v) for v in task[:7])
    ib = g.ib
    if kind == GETRF:
        F, pv = LU.getrf(g.tile(k, k), ib)
        g.tile(k, k)[:] = F
        g.piv[(k, k)] = pv
    elif kind == GESSM:
        C = g.slab(k, j, s)
        C[:] = LU.gessm(C, g.tile(k, k), g.piv[(k, k)], ib)
    elif kind == TSTRF:
        Ut, Lb, L1, pv = LU.tstrf(g.tile(k, k), g.tile(i, k), ib)
        g.tile(k, k)[:] = np.tril(g.tile(k, k), -1) + Ut
        g.tile(i, k)[:] = Lb
        g.piv[(i, k)] = pv
        g.L1[(i, k)] = L1
    elif kind == SSSSM:
        top, bot = g.slab(k, j, s), g.slab(i, j, s)
        t2, b2 = LU.ssssm(top, bot, g.tile(i, k), g.L1[(i, k)], g.piv[(i, k)], ib)
        top[:], bot[:] = t2, b2
    elif kind == TRSM_UPD:
        C = g.slab(k, j, s)
        C -= g.tile(k, l) @ g.slab(l, j, s)
    elif kind == TRSM_SOLVE:
        C = g.slab(k, j, s)
        nv = min(g.nb, g.n - k * g.nb)
        R = np.triu(g.tile(k, k))[:nv, :nv]
        X = np.array(C[:nv], copy=True)
        for r in range(nv - 1, -1, -1):
            X[r] = (X[r] - R[r, r + 1:] @ X[r + 1:]) / R[r, r]
        C[:nv] = X
        C[nv:] = 0.0
    else:
        raise AssertionError(kind)


def expected_lu_tasks(mode, g, trsm=0):
    out = []
    cols_all = range(g.q + g.qb)
    for k in range(g.kt):
        if mode == FACTOR:
            out.append((GETRF, 0, k, k, k, 0))
            out += [(TSTRF, 0, k, i, k, 0) for i in range(k + 1, g.p)]
        cols = [j for j in cols_all if j > k] if mode == FACTOR else [j for j in cols_all if j >= g.q]
        out += [(GESSM, s, k, k, j, 0) for j in cols for s in range(g.slabs(j))]
        out += [(SSSSM, s, k, i, j, 0) for i in range(k + 1, g.p) for j in cols for s in range(g.slabs(j))]
    if trsm:
        for j in range(g.q, g.q + g.qb):
            for s in range(g.slabs(j)):
                for k in range(g.kt):
                    out.append((TRSM_SOLVE, s, k, k, j, 0))
                    out += [(TRSM_UPD, s, k, k, j, l) for l in range(k + 1, g.kt)]
    return sorted(out)


def lu_plan(mode, g, trsm=0, workers=7, policy=-1):
    tasks, stats = tqr.tqr_debug_plan(LUF | mode, g.m, g.n, g.nb, g.ib, g.cs, g.nrhs, trsm, workers, policy)
    got = sorted((int(t[0]), int(t[1]), int(t[3]), int(t[4]), int(t[5]), int(t[6])) for t in tasks)
    assert got == expected_lu_tasks(mode, g, trsm)
    return tasks, stats


SHAPES = [(64, 64, 16, 4, 8), (70, 45, 16, 8, 16), (45, 70, 16, 4, 4), (33, 33, 8, 2, 8), (96, 40, 32, 8, 8)]


@pytest.mark.parametrize("m,n,nb,ib,cs", SHAPES)
@pytest.mark.parametrize("policy", [0, 1])
def test_lu_factor_plan_replays_the_oracle(m, n, nb, ib, cs, policy):
    A = inputs.normal_matrix(m, n, m + 2 * n)
    f = LU.tiled_lu(A, nb, ib)
    for seed in (None, 5):
        g = LuGrid(m, n, nb, ib, cs)
        g.A[:m, :n] = A
        plan, _ = lu_plan(FACTOR, g, policy=policy)
        check_order_satisfies_waits(LUF | FACTOR, g, plan)
        order = plan if seed is None else random_valid_order(LUF | FACTOR, g, plan, seed)
        for t in order:
            execute(g, t)
        # same kernels, same per-tile update sequence: identical bits
        assert np.array_equal(g.A, f.Ap)
        for key, pv in f.piv.items():
            assert np.array_equal(g.piv[key], pv)


@pytest.mark.parametrize("n,nb,ib,cs,nrhs", [(64, 16, 4, 8, 3), (45, 16, 8, 8, 17), (33, 8, 2, 4, 1)])
def test_lu_factor_and_solve_in_one_plan(n, nb, ib, cs, nrhs):
    A = inputs.normal_matrix(n, n, 21)
    B = inputs.normal_matrix(n, nrhs, 22)
    g = LuGrid(n, n, nb, ib, cs, nrhs)
    g.A[:n, :n] = A
    g.B[:n, :nrhs] = B
    plan, _ = lu_plan(FACTOR, g, trsm=1)
    check_order_satisfies_waits(LUF | FACTOR, g, plan)
    for t in random_valid_order(LUF | FACTOR, g, plan, 2):
        execute(g, t)
    X = g.B[:n, :nrhs]
    assert np.allclose(X, np.linalg.solve(A, B), atol=1e-9 * np.linalg.cond(A))


@pytest.mark.parametrize("n,nb,ib,cs,nrhs", [(64, 16, 4, 8, 3), (70, 16, 8, 16, 20), (40, 8, 8, 8, 1)])
def test_lu_solve_plan_on_existing_factors(n, nb, ib, cs, nrhs):
    A = inputs.normal_matrix(n, n, 31)
    B = inputs.normal_matrix(n, nrhs, 32)
    f = LU.tiled_lu(A, nb, ib)
    g = LuGrid(n, n, nb, ib, cs, nrhs)
    g.A[:] = f.Ap
    g.piv, g.L1 = dict(f.piv), dict(f.L1)
    g.B[:n, :nrhs] = B
    plan, _ = lu_plan(APPLY_QT, g, trsm=1)
    check_order_satisfies_waits(LUF | APPLY_QT, g, plan)
    for t in random_valid_order(LUF | APPLY_QT, g, plan, 3):
        execute(g, t)
    assert np.allclose(g.B[:n, :nrhs], LU.lu_solve(f, B), rtol=0, atol=1e-12 * np.abs(LU.lu_solve(f, B)).max())


def test_lu_plan_rejects_tree_and_other_modes():
    with pytest.raises(RuntimeError):
        tqr.tqr_debug_plan(LUF | FACTOR, 64, 64, 16, 4, 8, 0, 0, 7, -1, D=2)
    with pytest.raises(RuntimeError):
        tqr.tqr_debug_plan(LUF | 2, 64, 64, 16, 4, 8, 4, 0, 7, -1)


# 2b x b bottoms -------------------------------------------------------------
PAIR = 32
TSTRF2, SSSSM2 = 20, 21


def execute_pairs(g, task):
    kind, s, _, k, h, j, l = (int(v) for v in task[:7])
    if kind not in (TSTRF2, SSSSM2):
        return execute(g, task)
    ib = g.ib
    rows = list(range(h, h + l))
    if kind == TSTRF2:
        Ut, Lb, L1, pv = LU.tstrf(g.tile(k, k), np.vstack([g.tile(r, k) for r in rows]), ib)
        g.tile(k, k)[:] = np.tril(g.tile(k, k), -1) + Ut
        for a, r in enumerate(rows):
            g.tile(r, k)[:] = Lb[a * g.nb:(a + 1) * g.nb]
        g.piv[(h, k)] = pv
        g.L1[(h, k)] = L1
    else:
        top = g.slab(k, j, s)
        bots = [g.slab(r, j, s) for r in rows]
        Lb = np.vstack([g.tile(r, k) for r in rows])
        t2, b2 = LU.ssssm(top, np.vstack(bots), Lb, g.L1[(h, k)], g.piv[(h, k)], ib)
        top[:] = t2
        for a, b in enumerate(bots):
            b[:] = b2[a * g.nb:(a + 1) * g.nb]


@pytest.mark.parametrize("m,n,nb,ib,cs", SHAPES)
def test_lu_pair_factor_plan_replays_the_oracle(m, n, nb, ib, cs):
    A = inputs.normal_matrix(m, n, 3 * m + n)
    f = LU.tiled_lu_pairs(A, nb, ib)
    for seed in (None, 6):
        g = LuGrid(m, n, nb, ib, cs)
        g.A[:m, :n] = A
        plan, _ = tqr.tqr_debug_plan(PAIR | LUF | FACTOR, m, n, nb, ib, cs, 0, 0, 7, -1)
        check_order_satisfies_waits(PAIR | LUF | FACTOR, g, plan)
        kinds = {int(t[0]) for t in plan}
        assert kinds <= {13, 14, TSTRF2, SSSSM2} and (TSTRF2 in kinds or g.p == 1)
        for t in (plan if seed is None else random_valid_order(PAIR | LUF | FACTOR, g, plan, seed)):
            execute_pairs(g, t)
        assert np.array_equal(g.A, f.Ap)


@pytest.mark.parametrize("n,nb,ib,cs,nrhs", [(64, 16, 4, 8, 3), (45, 16, 8, 8, 17)])
def test_lu_pair_factor_and_solve_in_one_plan(n, nb, ib, cs, nrhs):
    A = inputs.normal_matrix(n, n, 24)
    B = inputs.normal_matrix(n, nrhs, 25)
    g = LuGrid(n, n, nb, ib, cs, nrhs)
    g.A[:n, :n] = A
    g.B[:n, :nrhs] = B
    plan, _ = tqr.tqr_debug_plan(PAIR | LUF | FACTOR, n, n, nb, ib, cs, nrhs, 1, 7, -1)
    check_order_satisfies_waits(PAIR | LUF | FACTOR, g, plan)
    for t in random_valid_order(PAIR | LUF | FACTOR, g, plan, 2):
        execute_pairs(g, t)
    assert np.allclose(g.B[:n, :nrhs], np.linalg.solve(A, B), atol=1e-9 * np.linalg.cond(A))
