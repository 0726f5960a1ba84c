"""Pins for the tiled LU oracle (pairwise pivoting, Section 5's LU analogue of
Algorithm 1).

The pins reach past the tiled code: one tile with ib = b is LAPACK's
partially pivoted LU (scipy's dgetrf as a third opinion); a column
diagonally dominant matrix never pivots, so its U is the unique LU factor
(computed here in exact rationals); the factorization's transformations
applied to A itself must give U with zeros below it; solves must match an
independent dense solver; a 2 x 2 case with 1 x 1 tiles is worked by hand;
planted mistakes must fail."""
from fractions import Fraction

import numpy as np
import pytest

from oracle import tiled_lu as LU
from paper_0707_3548_gb300 import inputs

U53 = 2.0 ** -53


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_hand_worked_2x2_with_1x1_tiles():
    # GETRF [1]; GESSM keeps [2]; TSTRF picks 3 over 1 (swap, multiplier 1/3);
    # SSSSM swaps 2 and 4 then 2 - 4/3; GETRF [2/3]
    f = LU.tiled_lu(np.array([[1.0, 2.0], [3.0, 4.0]]), 1, 1)
    assert f.piv[(1, 0)][0] == 0
    assert f.tile(1, 0)[0, 0] == 1.0 / 3.0
    assert np.allclose(f.U, [[3.0, 4.0], [0.0, 2.0 / 3.0]], rtol=0, atol=4 * U53)
    x = LU.lu_solve(f, np.array([5.0, 11.0]))
    assert np.allclose(x[:, 0], [1.0, 2.0], rtol=0, atol=8 * U53)


def test_single_tile_full_block_is_lapack_getrf():
    scipy_linalg = pytest.importorskip("scipy.linalg")
    for seed, b in ((1, 8), (2, 16), (3, 33)):
        A = inputs.normal_matrix(b, b, seed)
        F, piv = LU.getrf(A, b)
        lu, ipiv = scipy_linalg.lu_factor(A)
        assert np.array_equal(piv, ipiv)
        assert _rel(F, lu) <= 50 * b * U53


@pytest.mark.parametrize("b,ib", [(16, 4), (16, 8), (24, 8), (32, 1)])
def test_inner_blocking_keeps_pivots_and_u(b, ib):
    """Blocks change where multipliers sit, not the elimination: same pivots,
    same U, and the same operator on other columns."""
    A = inputs.normal_matrix(b, b, 4)
    F1, p1 = LU.getrf(A, b)
    Fb, pb = LU.getrf(A, ib)
    assert np.array_equal(p1, pb)
    assert _rel(np.triu(Fb), np.triu(F1)) <= 50 * b * U53
    C = inputs.normal_matrix(b, 5, 5)
    assert _rel(LU.gessm(C, Fb, pb, ib), LU.gessm(C, F1, p1, b)) <= 50 * b * U53
    U0 = np.triu(inputs.normal_matrix(b, b, 6))
    A2 = inputs.normal_matrix(b, b, 7)
    r1 = LU.tstrf(U0, A2, b)
    rb = LU.tstrf(U0, A2, ib)
    assert np.array_equal(r1[3], rb[3])
    assert _rel(rb[0], r1[0]) <= 50 * b * U53
    Ct, Cb = inputs.normal_matrix(b, 3, 8), inputs.normal_matrix(b, 3, 9)
    o1 = LU.ssssm(Ct, Cb, r1[1], r1[2], r1[3], b)
    ob = LU.ssssm(Ct, Cb, rb[1], rb[2], rb[3], ib)
    assert _rel(ob[0], o1[0]) <= 50 * b * U53 and _rel(ob[1], o1[1]) <= 50 * b * U53


def _doolittle_exact(A):
    n = len(A)
    M = [[Fraction(int(v)) for v in row] for row in A]
    for c in range(n):
        for r in range(c + 1, n):
            l = M[r][c] / M[c][c]
            for d in range(c, n):
                M[r][d] -= l * M[c][d]
    return np.array([[float(M[r][d]) if d >= r else 0.0 for d in range(n)] for r in range(n)])


@pytest.mark.parametrize("n,nb,ib", [(12, 4, 2), (13, 4, 4), (10, 3, 1)])
def test_diagonally_dominant_never_pivots_and_gives_the_unique_u(n, nb, ib):
    g = np.random.default_rng(n)
    A = g.integers(-9, 10, size=(n, n)).astype(np.float64)
    A += np.diag(np.abs(A).sum(axis=0) + 1.0)     # strictly column diagonally dominant
    f = LU.tiled_lu(A, nb, ib)
    for (i, k), pv in f.piv.items():
        if i == k:
            assert np.array_equal(pv, np.arange(nb))
        else:
            assert (pv == -1).all()
    assert _rel(f.U, _doolittle_exact(A)) <= 10 * n * U53


SHAPES = [(64, 64, 16, 4), (70, 70, 16, 8), (45, 45, 8, 2), (33, 33, 8, 8), (100, 60, 16, 4), (40, 90, 16, 8)]


@pytest.mark.parametrize("m,n,nb,ib", SHAPES)
def test_transformations_applied_to_a_give_u(m, n, nb, ib):
    A = inputs.normal_matrix(m, n, m + n)
    f = LU.tiled_lu(A, nb, ib)
    Y = LU.apply_linv(f, A)
    k = min(m, n)
    U = np.triu(f.Ap[:m, :n])
    assert _rel(Y[:k], U[:k]) <= 1e3 * n * U53          # pairwise pivoting growth stays modest here
    if m > n:
        assert np.linalg.norm(Y[n:]) <= 1e3 * n * U53 * np.linalg.norm(A)


@pytest.mark.parametrize("n,nb,ib", [(64, 16, 4), (70, 16, 8), (33, 8, 8), (96, 32, 8)])
def test_solve_matches_dense_solver(n, nb, ib):
    A = inputs.normal_matrix(n, n, 11 + n)
    B = inputs.normal_matrix(n, 3, 12)
    f = LU.tiled_lu(A, nb, ib)
    X = LU.lu_solve(f, B)
    Xd = np.linalg.solve(A, B)
    kappa = np.linalg.cond(A)
    assert _rel(X, Xd) <= 1e3 * kappa * n * U53
    assert np.linalg.norm(A @ X - B) / (np.linalg.norm(A) * np.linalg.norm(X)) <= 1e3 * n * U53


def test_zero_padding_leaves_factors_unchanged():
    A = inputs.normal_matrix(37, 37, 13)
    f = LU.tiled_lu(A, 8, 4)
    assert not f.Ap[37:].any() or np.allclose(f.Ap[37:, :37], 0.0)
    X = LU.lu_solve(f, np.eye(37))
    assert np.linalg.norm(A @ X - np.eye(37)) <= 1e3 * 37 * U53 * np.linalg.cond(A)


def test_planted_mistakes_fail_the_pins(monkeypatch):
    n, nb, ib = 48, 16, 4
    A = inputs.normal_matrix(n, n, 14)
    B = inputs.normal_matrix(n, 2, 15)
    good = LU.lu_solve(LU.tiled_lu(A, nb, ib), B)
    assert np.linalg.norm(A @ good - B) <= 1e-10 * np.linalg.norm(B)

    real_ssssm = LU.ssssm

    def ssssm_without_swaps(Ct, Cb, Lb, L1, piv, ib_):
        return real_ssssm(Ct, Cb, Lb, L1, np.full_like(piv, -1), ib_)

    monkeypatch.setattr(LU, "ssssm", ssssm_without_swaps)
    bad = LU.lu_solve(LU.tiled_lu(A, nb, ib), B)
    assert np.linalg.norm(A @ bad - B) > 1e-3 * np.linalg.norm(B)
    monkeypatch.setattr(LU, "ssssm", real_ssssm)

    real_solve = LU._block_solve

    def transposed_l11(L11, X):
        return real_solve(np.tril(L11.T, -1) + np.eye(L11.shape[0]), X)

    monkeypatch.setattr(LU, "_block_solve", transposed_l11)
    bad = LU.lu_solve(LU.tiled_lu(A, nb, ib), B)
    assert np.linalg.norm(A @ bad - B) > 1e-3 * np.linalg.norm(B)


def test_zero_diagonal_tile_takes_pivots_from_below():
    nb = 8
    Q = inputs.normal_matrix(nb, nb, 16) + 4 * np.eye(nb)
    A = np.block([[np.zeros((nb, nb)), np.eye(nb)], [Q, inputs.normal_matrix(nb, nb, 17)]])
    f = LU.tiled_lu(A, nb, 4)
    assert (f.piv[(1, 0)] >= 0).all()
    B = inputs.normal_matrix(2 * nb, 2, 18)
    X = LU.lu_solve(f, B)
    assert np.linalg.norm(A @ X - B) <= 1e-12 * np.linalg.norm(B) * np.linalg.cond(A)


# 2b x b bottoms -------------------------------------------------------------

@pytest.mark.parametrize("m,n,nb,ib", SHAPES)
def test_pair_transformations_applied_to_a_give_u(m, n, nb, ib):
    A = inputs.normal_matrix(m, n, m + 2 * n)
    f = LU.tiled_lu_pairs(A, nb, ib)
    Y = LU.pairs_apply_linv(f, A)
    k = min(m, n)
    U = np.triu(f.Ap[:m, :n])
    assert _rel(Y[:k], U[:k]) <= 1e3 * n * U53
    if m > n:
        assert np.linalg.norm(Y[n:]) <= 1e3 * n * U53 * np.linalg.norm(A)


@pytest.mark.parametrize("n,nb,ib", [(64, 16, 4), (70, 16, 8), (33, 8, 8), (96, 32, 8)])
def test_pair_solve_matches_dense_solver(n, nb, ib):
    A = inputs.normal_matrix(n, n, 21 + n)
    B = inputs.normal_matrix(n, 3, 22)
    f = LU.tiled_lu_pairs(A, nb, ib)
    X = LU.pairs_lu_solve(f, B)
    assert _rel(X, np.linalg.solve(A, B)) <= 1e3 * np.linalg.cond(A) * n * U53
    assert np.linalg.norm(A @ X - B) / (np.linalg.norm(A) * np.linalg.norm(X)) <= 1e3 * n * U53


def test_pair_diagonally_dominant_gives_the_unique_u():
    n = 13
    g = np.random.default_rng(3)
    A = g.integers(-9, 10, size=(n, n)).astype(np.float64)
    A += np.diag(np.abs(A).sum(axis=0) + 1.0)
    f = LU.tiled_lu_pairs(A, 3, 1)
    assert all((pv == -1).all() for (i, k), pv in f.piv.items() if i != k)
    assert _rel(f.U, _doolittle_exact(A)) <= 10 * n * U53


def test_pair_two_tile_rows_are_the_flat_factorization():
    A = inputs.normal_matrix(32, 40, 23)
    assert np.array_equal(LU.tiled_lu_pairs(A, 16, 4).Ap, LU.tiled_lu(A, 16, 4).Ap)
