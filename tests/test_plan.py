"""Host logic of the device scheduler, checked on the CPU.

The task lists the library would launch are fetched with tqr_debug_plan and
replayed here task by task with the oracle's tile kernels (column slab by
column slab), in the plan's order and in random orders that respect the
version waits.  The replays must reproduce the oracle's sequential results,
which pins the task set, the slab decomposition, the per-mode orders and the
wait/signal rules at once."""
import itertools

import numpy as np
import pytest

from oracle import householder as H
from oracle import lstsq as LS
from oracle import tiled as TL
from paper_0707_3548_gb300 import inputs, tqr

GEQRT, TSQRT, LARFB, SSRFB, LARFB_N, SSRFB_N, TRSM_UPD, TRSM_SOLVE, TRSMT_UPD, TRSMT_SOLVE = range(10)
FACTOR, APPLY_QT, APPLY_Q, TRSM, TRSMT, FORM_Q = range(6)


class Grid:
    """Padded A tiles (p x q) and right-hand-side tiles (p x qb), BDL-like."""

    def __init__(self, m, n, nb, ib, cs, nrhs=0):
        self.m, self.n, self.nb, self.ib, self.cs, self.nrhs = m, n, nb, ib, cs, nrhs
        self.p, self.q = -(-m // nb), -(-n // nb)
        self.kt = min(self.p, self.q)
        self.qb = -(-nrhs // nb) if nrhs else 0
        self.A = np.zeros((self.p * nb, self.q * nb))
        self.B = np.zeros((self.p * nb, max(1, self.qb) * nb))
        self.T = {}

    def tile(self, i, j):
        nb = self.nb
        if j < self.q:
            return self.A[i * nb:(i + 1) * nb, j * nb:(j + 1) * nb]
        jb = j - self.q
        return self.B[i * nb:(i + 1) * nb, jb * nb:(jb + 1) * nb]

    def slab(self, i, j, s):
        t = self.tile(i, j)
        w = self.cs
        if j >= self.q:
            c0 = (j - self.q) * self.nb + s * self.cs
            w = min(self.cs, self.nrhs - c0)
        return t[:, s * self.cs: s * self.cs + w]

    def slabs(self, j):
        if j < self.q:
            return self.nb // self.cs
        c0 = (j - self.q) * self.nb
        w = min(self.nb, self.nrhs - c0)
        return -(-w // self.cs) if w > 0 else 0


def execute(g, task):
    kind, s, _, k, i, j, l = (int(v) for v in task[:7])
    ib = g.ib
    if kind == GEQRT:
        F, T = TL.geqrt(g.tile(k, k), ib)
        g.tile(k, k)[:] = F
        g.T[(k, k)] = T
    elif kind == TSQRT:
        R, V, T = TL.tsqrt(g.tile(k, k), g.tile(i, k), ib)
        g.tile(k, k)[:] = R
        g.tile(i, k)[:] = V
        g.T[(i, k)] = T
    elif kind in (LARFB, LARFB_N):
        C = g.slab(k, j, s)
        C[:] = TL.larfb(C, g.tile(k, k), g.T[(k, k)], ib, trans=(kind == LARFB))
    elif kind in (SSRFB, SSRFB_N):
        top, bot = g.slab(k, j, s), g.slab(i, j, s)
        t2, b2 = TL.ssrfb(top, bot, g.tile(i, k), g.T[(i, k)], ib, trans=(kind == SSRFB))
        top[:], bot[:] = t2, b2
    elif kind == TRSM_UPD:
        C = g.slab(k, j, s)
        C -= g.tile(k, l) @ g.slab(l, j, s)
    elif kind == TRSMT_UPD:
        C = g.slab(k, j, s)
        C -= g.tile(l, k).T @ g.slab(l, j, s)
    elif kind in (TRSM_SOLVE, TRSMT_SOLVE):
        C = g.slab(k, j, s)
        nv = min(g.nb, g.n - k * g.nb)
        R = np.triu(g.tile(k, k))[:nv, :nv]
        if kind == TRSM_SOLVE:
            C[:nv] = LS.back_substitution(R, C[:nv])
        else:
            C[:nv] = LS.forward_substitution_rt(R, C[:nv])
        C[nv:] = 0.0
    else:
        raise AssertionError(kind)


def expected_tasks(mode, g, trsm=0):
    """Independent enumeration of the task set (Algorithm 1 + slabs)."""
    out = []
    cols_all = range(g.q + g.qb)
    for k in range(g.kt):
        if mode == FACTOR:
            out.append((GEQRT, 0, k, k, k, 0))
            out += [(TSQRT, 0, k, i, k, 0) for i in range(k + 1, g.p)]
        cols = [j for j in cols_all if j > k] if mode == FACTOR else [j for j in cols_all if j >= g.q]
        if mode in (FACTOR, APPLY_QT):
            out += [(LARFB, s, k, k, j, 0) for j in cols for s in range(g.slabs(j))]
            out += [(SSRFB, s, k, i, j, 0) for i in range(k + 1, g.p) for j in cols for s in range(g.slabs(j))]
        if mode == FORM_Q:
            cols = [j for j in cols if j - g.q >= k]
        if mode in (APPLY_Q, FORM_Q):
            out += [(LARFB_N, s, k, k, j, 0) for j in cols for s in range(g.slabs(j))]
            out += [(SSRFB_N, s, k, i, j, 0) for i in range(k + 1, g.p) for j in cols for s in range(g.slabs(j))]
    if mode == TRSM or (mode in (FACTOR, APPLY_QT) and trsm):
        for j in range(g.q, g.q + g.qb):
            for s in range(g.slabs(j)):
                for k in range(g.kt):
                    out.append((TRSM_SOLVE, s, k, k, j, 0))
                    out += [(TRSM_UPD, s, k, k, j, l) for l in range(k + 1, g.kt)]
    if mode == TRSMT:
        for j in range(g.q, g.q + g.qb):
            for s in range(g.slabs(j)):
                for k in range(g.kt):
                    out.append((TRSMT_SOLVE, s, k, k, j, 0))
                    out += [(TRSMT_UPD, s, k, k, j, l) for l in range(k)]
    return sorted(out)


def check_order_satisfies_waits(mode, g, plan):
    """Replaying version counters in list order: every wait is met by the
    tasks before it (so the list is a topological order of the DAG)."""
    ver = {}
    for t in plan:
        waits, sigs = tqr.tqr_debug_rules(mode, g.m, g.n, g.nb, g.ib, g.cs, g.nrhs, t[:7])
        for ctr, cnt, v in waits:
            for c in range(cnt):
                assert ver.get(ctr + c, 0) >= v, (t, ctr + c, v)
        for ctr, cnt in sigs:
            for c in range(cnt):
                ver[ctr + c] = ver.get(ctr + c, 0) + 1


def random_valid_order(mode, g, plan, seed):
    """A random schedule that only starts tasks whose waits are met."""
    rng = np.random.default_rng(seed)
    rules = [tqr.tqr_debug_rules(mode, g.m, g.n, g.nb, g.ib, g.cs, g.nrhs, t[:7]) for t in plan]
    ver = {}
    left = list(range(len(plan)))
    out = []
    while left:
        ready = [x for x in left if all(ver.get(c + d, 0) >= v for c, cnt, v in rules[x][0] for d in range(cnt))]
        assert ready
        x = ready[rng.integers(len(ready))]
        left.remove(x)
        out.append(plan[x])
        for c, cnt in rules[x][1]:
            for d in range(cnt):
                ver[c + d] = ver.get(c + d, 0) + 1
    return out


def plan_of(mode, g, trsm=0, workers=7, policy=-1):
    tasks, stats = tqr.tqr_debug_plan(mode, g.m, g.n, g.nb, g.ib, g.cs, g.nrhs, trsm, workers, policy)
    got = sorted((int(t[0]), int(t[1]), int(t[3]), int(t[4]), int(t[5]), int(t[6])) for t in tasks)
    assert got == expected_tasks(mode, g, trsm)
    return tasks, stats


FACTOR_SHAPES = [
    # m, n, nb, ib, cs
    (64, 64, 16, 4, 8),
    (70, 45, 16, 8, 16),
    (45, 70, 16, 4, 4),
    (33, 17, 8, 2, 8),
    (96, 40, 32, 8, 8),
]


@pytest.mark.parametrize("m,n,nb,ib,cs", FACTOR_SHAPES)
@pytest.mark.parametrize("policy", [0, 1, 2])
def test_factor_plan_replays_algorithm1(m, n, nb, ib, cs, policy):
    A = inputs.uniform_matrix(m, n, m + n)
    g = Grid(m, n, nb, ib, cs)
    g.A[:m, :n] = A
    plan, stats = plan_of(FACTOR, g, policy=policy)
    check_order_satisfies_waits(FACTOR, g, plan)
    for t in plan:
        execute(g, t)
    f = TL.tiled_qr(A, nb, ib)
    assert np.allclose(g.A, f.Ap, rtol=0, atol=1e-13 * np.abs(f.Ap).max())
    for key, T in f.T.items():
        assert np.allclose(g.T[key], T, rtol=0, atol=1e-13 * max(1.0, np.abs(T).max()))
    # simulated makespan bounds
    chosen, other, pol, edges, cp, work = stats
    assert int(pol) == policy
    assert cp <= chosen * (1 + 1e-9) and work / 7 <= chosen * (1 + 1e-9) and chosen <= work * (1 + 1e-9)


def test_random_schedules_are_bitwise_identical():
    m, n, nb, ib, cs = 48, 40, 16, 4, 8
    A = inputs.normal_matrix(m, n, 3)
    plan, _ = plan_of(FACTOR, Grid(m, n, nb, ib, cs))
    results = []
    for order in [plan] + [random_valid_order(FACTOR, Grid(m, n, nb, ib, cs), plan, seed) for seed in range(3)]:
        g = Grid(m, n, nb, ib, cs)
        g.A[:m, :n] = A
        for t in order:
            execute(g, t)
        results.append(g.A.copy())
    for r in results[1:]:
        assert np.array_equal(r, results[0])


@pytest.mark.parametrize("m,n,nb,ib,cs,nrhs", [(70, 45, 16, 8, 8, 3), (64, 64, 16, 4, 16, 20), (50, 16, 8, 8, 8, 1)])
def test_factor_with_rhs_and_back_substitution_solves_ls(m, n, nb, ib, cs, nrhs):
    A = inputs.normal_matrix(m, n, 5)
    B = inputs.normal_matrix(m, nrhs, 6)
    g = Grid(m, n, nb, ib, cs, nrhs)
    g.A[:m, :n] = A
    g.B[:m, :nrhs] = B
    plan, _ = plan_of(FACTOR, g, trsm=1)
    check_order_satisfies_waits(FACTOR, g, plan)
    for t in plan:
        execute(g, t)
    X = g.B[:n, :nrhs]
    assert np.allclose(X, LS.lstsq(A, B), atol=1e-11)


@pytest.mark.parametrize("m,n,nb,ib,cs,nrhs", [(70, 45, 16, 8, 8, 3), (45, 70, 16, 4, 16, 17), (64, 64, 16, 16, 8, 5)])
def test_apply_plans(m, n, nb, ib, cs, nrhs):
    A = inputs.normal_matrix(m, n, 7)
    B = inputs.normal_matrix(m, nrhs, 8)
    f = TL.tiled_qr(A, nb, ib)
    for mode, ref in ((APPLY_QT, TL.apply_qt(f, B)), (APPLY_Q, TL.apply_q(f, B))):
        g = Grid(m, n, nb, ib, cs, nrhs)
        g.A[:] = f.Ap
        g.T = dict(f.T)
        g.B[:m, :nrhs] = B
        plan, _ = plan_of(mode, g)
        check_order_satisfies_waits(mode, g, plan)
        for t in random_valid_order(mode, g, plan, 1):
            execute(g, t)
        assert np.allclose(g.B[:m, :nrhs], ref, atol=1e-12)


@pytest.mark.parametrize("m,n,nb,ib,cs,ncols", [(70, 45, 16, 8, 8, 45), (64, 64, 16, 4, 16, 64), (50, 16, 8, 8, 8, 50),
                                                 (45, 70, 16, 4, 8, 45), (80, 33, 16, 16, 16, 20), (40, 24, 8, 4, 4, 1)])
def test_form_q_plan_skips_identity_columns(m, n, nb, ib, cs, ncols):
    """Explicit Q: apply Q to [I; 0] while step k skips right-hand-side tile
    columns < k.  The skipped tiles are exact zeros under those reflectors,
    so the result must equal the oracle's Q columns."""
    A = inputs.normal_matrix(m, n, 17)
    f = TL.tiled_qr(A, nb, ib)
    ref = TL.orgqr(f, ncols)
    for order_seed in (None, 3):
        g = Grid(m, n, nb, ib, cs, ncols)
        g.A[:] = f.Ap
        g.T = dict(f.T)
        g.B[:m, :ncols] = np.eye(m, ncols)
        plan, _ = plan_of(FORM_Q, g)
        check_order_satisfies_waits(FORM_Q, g, plan)
        order = plan if order_seed is None else random_valid_order(FORM_Q, g, plan, order_seed)
        for t in order:
            execute(g, t)
        assert np.allclose(g.B[:m, :ncols], ref, rtol=0, atol=1e-13)
    full, _ = plan_of(APPLY_Q, Grid(m, n, nb, ib, cs, ncols))
    assert len(plan) < len(full) or g.kt == 1


def test_form_q_plan_rejects_pair_variant():
    with pytest.raises(Exception):
        tqr.tqr_debug_plan(32 | FORM_Q, 64, 64, 16, 4, 8, 16, 0, 7, -1)


@pytest.mark.parametrize("m,n,nb,ib,cs,nrhs", [(70, 45, 16, 8, 8, 3), (64, 64, 16, 4, 16, 17), (50, 16, 8, 8, 8, 1)])
def test_resident_factor_solve_plan(m, n, nb, ib, cs, nrhs):
    """Q^T B followed by back substitution on an existing factorization
    (the solve of a repeated matrix) as one plan."""
    A = inputs.normal_matrix(m, n, 15)
    B = inputs.normal_matrix(m, nrhs, 16)
    f = TL.tiled_qr(A, nb, ib)
    g = Grid(m, n, nb, ib, cs, nrhs)
    g.A[:] = f.Ap
    g.T = dict(f.T)
    g.B[:m, :nrhs] = B
    plan, _ = plan_of(APPLY_QT, g, trsm=1)
    check_order_satisfies_waits(APPLY_QT, g, plan)
    for t in random_valid_order(APPLY_QT, g, plan, 2):
        execute(g, t)
    assert np.allclose(g.B[:n, :nrhs], LS.lstsq(A, B), atol=1e-11)


@pytest.mark.parametrize("n,nb,cs,nrhs", [(45, 16, 8, 3), (64, 16, 16, 2), (20, 8, 8, 9)])
def test_triangular_solve_plans(n, nb, cs, nrhs):
    A = inputs.normal_matrix(n + 10, n, 9)
    f = TL.tiled_qr(A, nb, 4)
    R = f.R[:n, :n]
    Bv = inputs.normal_matrix(n, nrhs, 10)
    for mode, ref in ((TRSM, LS.back_substitution(R, Bv)), (TRSMT, LS.forward_substitution_rt(R, Bv))):
        g = Grid(n + 10, n, nb, 4, cs, nrhs)
        g.A[:] = f.Ap
        g.B[:n, :nrhs] = Bv
        plan, _ = plan_of(mode, g)
        check_order_satisfies_waits(mode, g, plan)
        for t in plan:
            execute(g, t)
        assert np.allclose(g.B[:n, :nrhs], ref, atol=1e-10 * np.abs(ref).max())


def test_bottom_level_policy_no_worse_in_simulation_for_wide_dag():
    g = Grid(2048, 2048, 128, 32, 32)
    _, s0 = plan_of(FACTOR, g, workers=304, policy=0)
    _, s1 = plan_of(FACTOR, g, workers=304, policy=1)
    _, sb = plan_of(FACTOR, g, workers=304, policy=-1)
    assert sb[0] == min(s0[0], s1[0])


@pytest.mark.parametrize("m,n,nb,ib,cs,D", [(2048, 2048, 128, 32, 32, 0), (4096, 512, 64, 16, 16, 0),
                                            (4096, 512, 64, 16, 16, 4), (8192, 1024, 128, 16, 32, 2),
                                            (700, 500, 64, 16, 16, 0)])
def test_one_pass_critical_path_equals_bottom_level(m, n, nb, ib, cs, D):
    """The estimate used to choose the tree's domain size (one forward pass,
    every wait on the preceding writer) equals the longest path of the DAG
    built from the same rules; the work is the sum of the task costs."""
    cp, work = tqr.tqr_debug_critical_path(FACTOR, m, n, nb, ib, cs, D=D)
    _, st = tqr.tqr_debug_plan(FACTOR, m, n, nb, ib, cs, 0, 0, 304, 2, D=D)
    assert abs(cp - st[4]) <= 1e-9 * st[4]
    assert abs(work - st[5]) <= 1e-9 * st[5]
