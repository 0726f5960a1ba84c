"""Host logic of the 2b x b bottom variant, checked on the CPU: the library's
task lists (tqr_debug_plan with the pair flag) are replayed slab by slab with
the oracle's kernels, in plan order and in random orders that respect the
version waits, and must reproduce the oracle's pair factorization and its
Q^T B, Q B and least-squares solves."""
import numpy as np
import pytest

from oracle import lstsq as LS
from oracle import tiled as TL
from paper_0707_3548_gb300 import inputs, tqr
from tests.test_plan import (APPLY_Q, APPLY_QT, FACTOR, GEQRT, LARFB, LARFB_N, TRSM_SOLVE, TRSM_UPD, Grid,
                             check_order_satisfies_waits, random_valid_order)

PAIR = 32
TSQRT2, SSRFB2, SSRFB2_N = 17, 18, 19


def execute(g, task):
    kind, s, _, k, h, j, l = (int(v) for v in task[:7])
    ib = g.ib
    rows = list(range(h, h + l))
    if kind == GEQRT:
        F, T = TL.geqrt(g.tile(k, k), ib)
        g.tile(k, k)[:] = F
        g.T[(k, k)] = T
    elif kind in (LARFB, LARFB_N):
        C = g.slab(k, j, s)
        C[:] = TL.larfb(C, g.tile(k, k), g.T[(k, k)], ib, trans=(kind == LARFB))
    elif kind == TSQRT2:
        R, V, T = TL.tsqrt(g.tile(k, k), np.vstack([g.tile(r, k) for r in rows]), ib)
        g.tile(k, k)[:] = R
        for a, r in enumerate(rows):
            g.tile(r, k)[:] = V[a * g.nb:(a + 1) * g.nb]
        g.T[(h, k)] = T
    elif kind in (SSRFB2, SSRFB2_N):
        top = g.slab(k, j, s)
        bots = [g.slab(r, j, s) for r in rows]
        V = np.vstack([g.tile(r, k) for r in rows])
        t2, b2 = TL.ssrfb(top, np.vstack(bots), V, g.T[(h, k)], ib, trans=(kind == SSRFB2))
        top[:] = t2
        for a, b in enumerate(bots):
            b[:] = b2[a * g.nb:(a + 1) * g.nb]
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


def expected(mode, g, trsm=0):
    out = []
    for k in range(g.kt):
        cols = [j for j in range(g.q + g.qb) if (j > k if mode == FACTOR else j >= g.q)]
        if mode == FACTOR:
            out.append((GEQRT, 0, k, k, k, 0))
        lar = LARFB_N if mode == APPLY_Q else LARFB
        ss = SSRFB2_N if mode == APPLY_Q else SSRFB2
        out += [(lar, s, k, k, j, 0) for j in cols for s in range(g.slabs(j))]
        for h in range(k + 1, g.p, 2):
            l = 2 if h + 1 < g.p else 1
            if mode == FACTOR:
                out.append((TSQRT2, 0, k, h, k, l))
            out += [(ss, s, k, h, j, l) for j in cols for s in range(g.slabs(j))]
    if trsm:
        for j in range(g.q, g.q + g.qb):
            for s in range(g.slabs(j)):
                for k in range(g.kt):
                    out.append((TRSM_SOLVE, s, k, k, j, 0))
                    out += [(TRSM_UPD, s, k, k, j, l) for l in range(k + 1, g.kt)]
    return sorted(out)


def pair_plan(mode, g, trsm=0, policy=-1):
    tasks, stats = tqr.tqr_debug_plan(PAIR | mode, g.m, g.n, g.nb, g.ib, g.cs, g.nrhs, trsm, 7, policy)
    got = sorted((int(t[0]), int(t[1]), int(t[3]), int(t[4]), int(t[5]), int(t[6])) for t in tasks)
    assert got == expected(mode, g, trsm)
    check_order_satisfies_waits(PAIR | mode, g, tasks)
    return tasks


SHAPES = [(96, 48, 16, 4, 8), (100, 60, 16, 8, 16), (64, 64, 16, 16, 8), (150, 40, 16, 4, 4), (33, 17, 8, 2, 8),
          (70, 90, 16, 8, 8)]


@pytest.mark.parametrize("m,n,nb,ib,cs", SHAPES)
@pytest.mark.parametrize("policy", [-1, 2])
def test_pair_factor_plan_replays_the_oracle(m, n, nb, ib, cs, policy):
    A = inputs.normal_matrix(m, n, m + n)
    f = TL.tiled_qr_pairs(A, nb, ib)
    for seed in (None, 4):
        g = Grid(m, n, nb, ib, cs)
        g.A[:m, :n] = A
        plan = pair_plan(FACTOR, g, policy=policy)
        for t in (plan if seed is None else random_valid_order(PAIR | FACTOR, g, plan, seed)):
            execute(g, t)
        assert np.array_equal(g.A, f.Ap)


@pytest.mark.parametrize("m,n,nb,ib,cs,nrhs", [(96, 48, 16, 4, 8, 3), (70, 90, 16, 8, 16, 20), (150, 40, 16, 4, 4, 1)])
def test_pair_apply_plans(m, n, nb, ib, cs, nrhs):
    A = inputs.normal_matrix(m, n, 9)
    B = inputs.normal_matrix(m, nrhs, 10)
    f = TL.tiled_qr_pairs(A, nb, ib)
    for mode, ref in ((APPLY_QT, TL.pairs_apply_qt(f, B)), (APPLY_Q, TL.pairs_apply_q(f, B))):
        g = Grid(m, n, nb, ib, cs, nrhs)
        g.A[:] = f.Ap
        g.T = dict(f.T)
        g.B[:m, :nrhs] = B
        plan = pair_plan(mode, g)
        for t in random_valid_order(PAIR | mode, g, plan, 1):
            execute(g, t)
        assert np.allclose(g.B[:m, :nrhs], ref, rtol=0, atol=1e-12)


@pytest.mark.parametrize("m,n,nb,ib,cs,nrhs", [(96, 48, 16, 4, 8, 3), (150, 40, 16, 8, 16, 2)])
def test_pair_factor_and_least_squares_in_one_plan(m, n, nb, ib, cs, nrhs):
    A = inputs.normal_matrix(m, n, 11)
    B = inputs.normal_matrix(m, nrhs, 12)
    g = Grid(m, n, nb, ib, cs, nrhs)
    g.A[:m, :n] = A
    g.B[:m, :nrhs] = B
    plan = pair_plan(FACTOR, g, trsm=1)
    for t in random_valid_order(PAIR | FACTOR, g, plan, 2):
        execute(g, t)
    assert np.allclose(g.B[:n, :nrhs], LS.lstsq(A, B), atol=1e-11)
