"""Pins for the reduction-tree variant of the tiled oracle."""
import numpy as np
import pytest

from oracle import householder as H
from oracle import tiled as TL
from paper_0707_3548_gb300 import inputs

U53 = 2.0 ** -53


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_tree_merges_cover_every_head_once():
    for H_ in range(1, 20):
        heads = list(range(0, 3 * H_, 3))
        merges = TL.tree_merges(heads)
        eliminated = [b for _, _, b in merges]
        assert sorted(eliminated) == heads[1:]            # every head but the root, once
        alive = set(heads)
        for _, a, b in merges:
            assert a in alive and b in alive               # both still unmerged
            alive.discard(b)
        assert alive == {heads[0]}


def test_ttqrt_gives_triangular_v_and_matches_stacked_qr():
    nb, ib = 16, 4
    R1 = np.triu(inputs.uniform_matrix(nb, nb, 1))
    R2 = np.triu(inputs.uniform_matrix(nb, nb, 2))
    R, V, T = TL.ttqrt(R1, R2, ib)
    assert np.array_equal(V, np.triu(V))                  # exact zeros below the diagonal
    F, _ = H.geqr2(np.vstack([R1, R2]))
    assert _rel(H.sign_normalize(np.triu(R)), H.sign_normalize(H.r_factor(F)[:nb])) <= 1e-13


@pytest.mark.parametrize("m,n,nb,ib,D", [(160, 48, 16, 4, 1), (160, 48, 16, 8, 2), (150, 40, 16, 4, 3),
                                          (96, 96, 16, 4, 2), (70, 45, 16, 8, 1), (33, 17, 8, 2, 2)])
def test_tree_r_equals_unblocked_and_invariants(m, n, nb, ib, D):
    A = inputs.normal_matrix(m, n, 10 * m + n + D)
    f = TL.tree_qr(A, nb, ib, D)
    k = min(m, n)
    Ru = H.sign_normalize(H.r_factor(H.geqr2(A)[0]))[:k]
    assert _rel(H.sign_normalize(f.R)[:k], Ru) <= 1e-13
    Q = TL.tree_apply_q(f, np.eye(m))
    tol = 10 * max(m, n) * U53
    assert _rel(Q @ f.R, A) <= tol
    assert np.linalg.norm(np.eye(m) - Q.T @ Q) <= tol
    assert _rel(TL.tree_apply_qt(f, A), f.R) <= tol
    assert not f.Ap[m:, :].any()


def test_one_domain_is_algorithm_1_exactly():
    A = inputs.uniform_matrix(100, 60, 7)
    f = TL.tree_qr(A, 16, 4, D=100)
    g = TL.tiled_qr(A, 16, 4)
    assert np.array_equal(f.Ap, g.Ap)
    for key in g.T:
        assert np.array_equal(f.T[key], g.T[key])
    assert not f.T2


def test_mutation_untransposed_tt_apply_is_caught(monkeypatch):
    orig = TL.ssrfb

    def bad(Akj, Aij, Vik, Tik, ib, trans=True):
        if np.array_equal(Vik, np.triu(Vik)) and np.any(Vik):   # a TT merge: apply Q, not Q^T
            return orig(Akj, Aij, Vik, Tik, ib, trans=not trans)
        return orig(Akj, Aij, Vik, Tik, ib, trans)
    A = inputs.normal_matrix(96, 40, 3)
    monkeypatch.setattr(TL, "ssrfb", bad)
    f = TL.tree_qr(A, 16, 4, 1)
    Ru = H.sign_normalize(H.r_factor(H.geqr2(A)[0]))[:40]
    assert _rel(H.sign_normalize(f.R)[:40], Ru) > 1e-8
