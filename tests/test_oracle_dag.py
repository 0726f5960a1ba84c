"""Pins for the task set / DAG / operation count of Algorithm 1."""
import itertools

import pytest

from oracle import dag as D


@pytest.mark.parametrize("p,q", [(1, 1), (3, 3), (5, 3), (3, 5), (8, 8)])
def test_task_counts_per_step(p, q):
    # Section 3.2: per step one GEQRT, q-k LARFB, p-k TSQRT, (p-k)(q-k) SSRFB
    # (k counted from 1 there; 0-based step s has k = s + 1)
    for s, c in enumerate(D.counts_per_step(p, q)):
        k = s + 1
        assert c == {D.GEQRT: 1, D.LARFB: q - k, D.TSQRT: p - k, D.SSRFB: (p - k) * (q - k)}


def test_opcount_tends_to_five_halves():
    # Eq. opcount: total ~ 5/2 n^2 (m - n/3), i.e. 25% above 2 n^2 (m - n/3)
    for p, q in ((200, 200), (400, 100)):
        b = 1.0
        ratio = D.opcount_tiles(p, q) * b ** 3 / D.lapack_flops(p * b, q * b)
        assert ratio == pytest.approx(1.25, rel=0.02)


def _listed_edges(p, q):
    """The dependency list written independently from the kernels' read/write
    sets: GEQRT(k) <- SSRFB(k-1,k,k); LARFB(k,j) <- GEQRT(k), SSRFB(k-1,k,j);
    TSQRT(k,i) <- TSQRT(k,i-1) or GEQRT(k), SSRFB(k-1,i,k);
    SSRFB(k,i,j) <- TSQRT(k,i), LARFB(k,j) or SSRFB(k,i-1,j), SSRFB(k-1,i,j)."""
    E = set()
    for k in range(min(p, q)):
        if k > 0:
            E.add(((D.SSRFB, k - 1, k, k), (D.GEQRT, k, k, k)))
        for j in range(k + 1, q):
            E.add(((D.GEQRT, k, k, k), (D.LARFB, k, k, j)))
            if k > 0:
                E.add(((D.SSRFB, k - 1, k, j), (D.LARFB, k, k, j)))
        for i in range(k + 1, p):
            prev = (D.GEQRT, k, k, k) if i == k + 1 else (D.TSQRT, k, i - 1, k)
            E.add((prev, (D.TSQRT, k, i, k)))
            if k > 0:
                E.add(((D.SSRFB, k - 1, i, k), (D.TSQRT, k, i, k)))
            for j in range(k + 1, q):
                E.add(((D.TSQRT, k, i, k), (D.SSRFB, k, i, j)))
                prevw = (D.LARFB, k, k, j) if i == k + 1 else (D.SSRFB, k, i - 1, j)
                E.add((prevw, (D.SSRFB, k, i, j)))
                if k > 0:
                    E.add(((D.SSRFB, k - 1, i, j), (D.SSRFB, k, i, j)))
    return E


@pytest.mark.parametrize("p,q", [(2, 2), (3, 3), (4, 2), (2, 4), (4, 4)])
def test_dataflow_dag_matches_dependency_list(p, q):
    red = D.reduced_edges(p, q)
    listed = _listed_edges(p, q)
    # every listed edge is implied by the data-flow DAG, and the data-flow
    # DAG's minimal edges are all listed
    full = D.edges(p, q)
    assert red <= listed
    reach = _closure(full, D.tasks(p, q))
    for a, b in listed:
        assert b in reach[a]


def _closure(E, order):
    succ = {}
    for a, b in E:
        succ.setdefault(a, set()).add(b)
    reach = {}
    for t in reversed(order):
        r = set()
        for s in succ.get(t, ()):
            r.add(s)
            r |= reach[s]
        reach[t] = r
    return reach


def test_subdag_property():
    # Section 3.3: for p1 >= p2, q1 >= q2 the p2 x q2 DAG is a subgraph of
    # the p1 x q1 DAG
    for (p1, q1), (p2, q2) in [((4, 4), (3, 3)), ((5, 3), (4, 2)), ((4, 5), (2, 5))]:
        assert set(D.tasks(p2, q2)) <= set(D.tasks(p1, q1))
        assert D.reduced_edges(p2, q2) <= D.edges(p1, q1)


def test_priorities_order():
    # Section 3.3: GEQRT > TSQRT > LARFB > SSRFB
    order = sorted(D.PRIORITY, key=D.PRIORITY.get)
    assert order == [D.GEQRT, D.TSQRT, D.LARFB, D.SSRFB]


def test_algorithm1_order_is_topological():
    for p, q in ((4, 4), (5, 2), (2, 5)):
        order = D.tasks(p, q)
        pos = {t: n for n, t in enumerate(order)}
        for a, b in D.edges(p, q):
            assert pos[a] < pos[b]


def test_critical_path_single_tile_column():
    # p x 1: GEQRT then a chain of p-1 TSQRTs
    assert D.critical_path(5, 1) == pytest.approx(2.0 + 4 * 10.0 / 3.0)
