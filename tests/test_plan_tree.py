"""Host logic of the reduction-tree variant, replayed on the CPU with the
oracle's tile kernels (see test_plan.py for the flat variant)."""
import numpy as np
import pytest

from oracle import lstsq as LS
from oracle import tiled as TL
from paper_0707_3548_gb300 import inputs, tqr
from tests.test_plan import Grid

(GEQRT, TSQRT, LARFB, SSRFB, LARFB_N, SSRFB_N, TRSM_UPD, TRSM_SOLVE, TRSMT_UPD, TRSMT_SOLVE,
 TTQRT, TTMQR, TTMQR_N) = range(13)
FACTOR, APPLY_QT, APPLY_Q = range(3)


class TreeGrid(Grid):
    def __init__(self, *a, **kw):
        super().__init__(*a, **kw)
        self.T2 = {}


def execute(g, task):
    kind, s, _, k, i, j, l = (int(v) for v in task[:7])
    ib = g.ib
    if kind == GEQRT:
        F, T = TL.geqrt(g.tile(i, k), ib)
        g.tile(i, k)[:] = F
        g.T[(i, k)] = T
    elif kind in (LARFB, LARFB_N):
        C = g.slab(i, j, s)
        C[:] = TL.larfb(C, g.tile(i, k), g.T[(i, k)], ib, trans=(kind == LARFB))
    elif kind == TSQRT:
        R, V, T = TL.tsqrt(g.tile(l, k), g.tile(i, k), ib)
        g.tile(l, k)[:] = R
        g.tile(i, k)[:] = V
        g.T[(i, k)] = T
    elif kind in (SSRFB, SSRFB_N):
        top, bot = g.slab(l, j, s), g.slab(i, j, s)
        t2, b2 = TL.ssrfb(top, bot, g.tile(i, k), g.T[(i, k)], ib, trans=(kind == SSRFB))
        top[:], bot[:] = t2, b2
    elif kind == TTQRT:
        R, V, T = TL.ttqrt(g.tile(l, k), g.tile(i, k), ib)
        g.tile(l, k)[:] = R
        g.tile(i, k)[:] = np.tril(g.tile(i, k), -1) + np.triu(V)
        g.T2[(i, k)] = T
    elif kind in (TTMQR, TTMQR_N):
        top, bot = g.slab(l, j, s), g.slab(i, j, s)
        t2, b2 = TL.ssrfb(top, bot, np.triu(g.tile(i, k)), g.T2[(i, k)], ib, trans=(kind == TTMQR))
        top[:], bot[:] = t2, b2
    elif kind == TRSM_UPD:
        C = g.slab(k, j, s)
        C -= g.tile(k, l) @ g.slab(l, j, s)
    elif kind == TRSM_SOLVE:
        C = g.slab(k, j, s)
        nv = min(g.nb, g.n - k * g.nb)
        C[:nv] = LS.back_substitution(np.triu(g.tile(k, k))[:nv, :nv], C[:nv])
        C[nv:] = 0.0
    else:
        raise AssertionError(kind)


def rules(mode, g, t, D):
    return tqr.tqr_debug_rules(mode, g.m, g.n, g.nb, g.ib, g.cs, g.nrhs, t[:7], D=D)


def check_order(mode, g, plan, D):
    ver = {}
    for t in plan:
        waits, sigs = rules(mode, g, t, D)
        for ctr, cnt, v in waits:
            for c in range(cnt):
                assert ver.get(ctr + c, 0) >= v, (t, ctr + c, v)
        for ctr, cnt in sigs:
            for c in range(cnt):
                ver[ctr + c] = ver.get(ctr + c, 0) + 1


def random_order(mode, g, plan, D, seed):
    rng = np.random.default_rng(seed)
    rl = [rules(mode, g, t, D) for t in plan]
    ver, left, out = {}, list(range(len(plan))), []
    while left:
        ready = [x for x in left if all(ver.get(c + d, 0) >= v for c, cnt, v in rl[x][0] for d in range(cnt))]
        assert ready
        x = ready[rng.integers(len(ready))]
        left.remove(x)
        out.append(plan[x])
        for c, cnt in rl[x][1]:
            for d in range(cnt):
                ver[c + d] = ver.get(c + d, 0) + 1
    return out


def expected_factor_tasks(g, D):
    out = []
    cols = range(g.q + g.qb)
    for k in range(g.kt):
        heads = TL.tree_heads(k, g.p, D)
        for h in heads:
            out.append((GEQRT, 0, k, h, k, 0))
            out += [(LARFB, s, k, h, j, 0) for j in cols if j > k for s in range(g.slabs(j))]
            for i in range(h + 1, min(h + D, g.p)):
                out.append((TSQRT, 0, k, i, k, h))
                out += [(SSRFB, s, k, i, j, h) for j in cols if j > k for s in range(g.slabs(j))]
        for _, a, b in TL.tree_merges(heads):
            out.append((TTQRT, 0, k, b, k, a))
            out += [(TTMQR, s, k, b, j, a) for j in cols if j > k for s in range(g.slabs(j))]
    return sorted(out)


SHAPES = [(160, 48, 16, 4, 8, 1), (160, 48, 16, 8, 16, 2), (150, 40, 16, 4, 8, 3), (96, 96, 16, 4, 16, 2),
          (70, 45, 16, 8, 8, 1), (33, 17, 8, 2, 8, 2)]


@pytest.mark.parametrize("m,n,nb,ib,cs,D", SHAPES)
def test_tree_factor_plan_replays_oracle(m, n, nb, ib, cs, D):
    A = inputs.normal_matrix(m, n, m + 7 * D)
    ref = TL.tree_qr(A, nb, ib, D)
    for policy in (0, 1):
        g = TreeGrid(m, n, nb, ib, cs)
        g.A[:m, :n] = A
        plan, _ = tqr.tqr_debug_plan(FACTOR, m, n, nb, ib, cs, 0, 0, workers=7, policy=policy, D=D)
        got = sorted((int(t[0]), int(t[1]), int(t[3]), int(t[4]), int(t[5]), int(t[6])) for t in plan)
        assert got == expected_factor_tasks(g, D)
        check_order(FACTOR, g, plan, D)
        for t in plan:
            execute(g, t)
        assert np.allclose(g.A, ref.Ap, rtol=0, atol=1e-13 * np.abs(ref.Ap).max())
        for key, T in ref.T2.items():
            assert np.allclose(g.T2[key], T, atol=1e-13 * max(1, np.abs(T).max()))


def test_tree_random_schedules_bitwise_equal():
    m, n, nb, ib, cs, D = 128, 40, 16, 4, 8, 2
    A = inputs.normal_matrix(m, n, 1)
    plan, _ = tqr.tqr_debug_plan(FACTOR, m, n, nb, ib, cs, 0, 0, workers=5, D=D)
    outs = []
    for order in [plan] + [random_order(FACTOR, TreeGrid(m, n, nb, ib, cs), plan, D, sd) for sd in range(3)]:
        g = TreeGrid(m, n, nb, ib, cs)
        g.A[:m, :n] = A
        for t in order:
            execute(g, t)
        outs.append(g.A.copy())
    for o in outs[1:]:
        assert np.array_equal(o, outs[0])


@pytest.mark.parametrize("m,n,nb,ib,cs,nrhs,D", [(160, 48, 16, 4, 8, 3, 1), (150, 40, 16, 8, 8, 17, 3),
                                                 (96, 96, 16, 4, 16, 2, 2)])
def test_tree_apply_and_solve_plans(m, n, nb, ib, cs, nrhs, D):
    A = inputs.normal_matrix(m, n, 3)
    B = inputs.normal_matrix(m, nrhs, 4)
    f = TL.tree_qr(A, nb, ib, D)
    for mode, trsm, ref in ((APPLY_QT, 0, TL.tree_apply_qt(f, B)), (APPLY_Q, 0, TL.tree_apply_q(f, B)),
                            (APPLY_QT, 1, None)):
        g = TreeGrid(m, n, nb, ib, cs, nrhs)
        g.A[:] = f.Ap
        g.T = dict(f.T)
        g.T2 = dict(f.T2)
        g.B[:m, :nrhs] = B
        plan, _ = tqr.tqr_debug_plan(mode, m, n, nb, ib, cs, nrhs, trsm, workers=5, D=D)
        check_order(mode, g, plan, D)
        for t in random_order(mode, g, plan, D, 1):
            execute(g, t)
        if ref is not None:
            assert np.allclose(g.B[:m, :nrhs], ref, atol=1e-12)
        else:
            assert np.allclose(g.B[:n, :nrhs], LS.lstsq(A, B), atol=1e-11)


def test_tree_factor_with_rhs_and_solve():
    m, n, nb, ib, cs, nrhs, D = 150, 40, 16, 4, 8, 5, 2
    A = inputs.normal_matrix(m, n, 8)
    B = inputs.normal_matrix(m, nrhs, 9)
    g = TreeGrid(m, n, nb, ib, cs, nrhs)
    g.A[:m, :n] = A
    g.B[:m, :nrhs] = B
    plan, _ = tqr.tqr_debug_plan(FACTOR, m, n, nb, ib, cs, nrhs, 1, workers=6, D=D)
    check_order(FACTOR, g, plan, D)
    for t in plan:
        execute(g, t)
    assert np.allclose(g.B[:n, :nrhs], LS.lstsq(A, B), atol=1e-11)


def test_tree_shortens_simulated_critical_path_for_tall_skinny():
    flat = tqr.tqr_debug_plan(FACTOR, 65536, 2048, 128, 16, 32, 0, 0, workers=304, D=0)[1]
    tree = tqr.tqr_debug_plan(FACTOR, 65536, 2048, 128, 16, 32, 0, 0, workers=304, D=32)[1]
    assert tree[4] < 0.6 * flat[4]       # critical path
    assert tree[0] < flat[0]             # simulated makespan


@pytest.mark.parametrize("m,n,nb,ib,cs,ncols,D", [(160, 48, 16, 4, 8, 48, 1), (150, 40, 16, 8, 8, 150, 3),
                                                  (96, 96, 16, 4, 16, 96, 2), (200, 60, 16, 8, 16, 37, 4)])
def test_tree_explicit_q_plan_skips_identity_columns(m, n, nb, ib, cs, ncols, D):
    A = inputs.normal_matrix(m, n, 5)
    f = TL.tree_qr(A, nb, ib, D)
    g = TreeGrid(m, n, nb, ib, cs, ncols)
    g.A[:] = f.Ap
    g.T = dict(f.T)
    g.T2 = dict(f.T2)
    g.B[:m, :ncols] = np.eye(m, ncols)
    plan, _ = tqr.tqr_debug_plan(5, m, n, nb, ib, cs, ncols, 0, workers=5, D=D)
    full, _ = tqr.tqr_debug_plan(APPLY_Q, m, n, nb, ib, cs, ncols, 0, workers=5, D=D)
    assert len(plan) < len(full) or g.kt == 1
    check_order(5, g, plan, D)
    for t in random_order(5, g, plan, D, 2):
        execute(g, t)
    assert np.allclose(g.B[:m, :ncols], TL.orgqr(f, ncols), rtol=0, atol=1e-13)
