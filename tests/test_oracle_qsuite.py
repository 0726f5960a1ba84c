"""Pins for the oracle's Q suite: op(Q) C, C op(Q) and the explicit columns of
Q (the DORMQR / DORGQR pair named in the paper's conclusion).

The pins reach past the tiled code: the thin Q of a full-rank matrix is unique
once R's diagonal signs are fixed, so it must match the unblocked Householder
oracle's Q (itself pinned by closed forms and exact cases); the right-hand
forms must match dense products with the formed Q; Q must be orthogonal and
reproduce A."""
import numpy as np
import pytest

from oracle import householder as H
from oracle import tiled as TL
from paper_0707_3548_gb300 import inputs

U53 = 2.0 ** -53


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _factor(m, n, nb, ib, D, seed):
    A = inputs.normal_matrix(m, n, seed)
    f = TL.tree_qr(A, nb, ib, D) if D else TL.tiled_qr(A, nb, ib)
    return A, f


SHAPES = [(64, 64, 16, 4, 0), (70, 45, 16, 8, 0), (45, 45, 8, 2, 0), (100, 30, 16, 16, 0),
          (160, 48, 16, 4, 2), (150, 40, 16, 8, 1)]


@pytest.mark.parametrize("m,n,nb,ib,D", SHAPES)
def test_thin_q_matches_unblocked_householder_q(m, n, nb, ib, D):
    A, f = _factor(m, n, nb, ib, D, 1)
    Qt = TL.orgqr(f, n)
    F, tau = H.geqr2(A)
    Qu = H.form_q(F, tau)[:, :n]
    s = np.sign(np.diag(f.R)[:n]) * np.sign(np.diag(H.r_factor(F))[:n])
    assert _rel(Qt, Qu * s) <= 50 * n * U53


@pytest.mark.parametrize("m,n,nb,ib,D", SHAPES)
def test_formed_q_is_orthogonal_and_reproduces_a(m, n, nb, ib, D):
    A, f = _factor(m, n, nb, ib, D, 2)
    Q = TL.orgqr(f, m)
    assert np.linalg.norm(Q.T @ Q - np.eye(m)) <= 10 * m * U53
    R = np.zeros((m, n))
    k = min(m, n)
    R[:k] = f.R[:k]
    assert _rel(Q @ R, A) <= 10 * n * U53
    # the leading columns do not depend on how many are formed
    for c in (0, 1, min(n, m), m):
        assert np.array_equal(TL.orgqr(f, c), Q[:, :c]) or _rel(TL.orgqr(f, c), Q[:, :c]) <= 4 * U53


@pytest.mark.parametrize("m,n,nb,ib,D", SHAPES)
@pytest.mark.parametrize("trans", ["N", "T"])
def test_ormqr_both_sides_match_dense_products(m, n, nb, ib, D, trans):
    A, f = _factor(m, n, nb, ib, D, 3)
    Q = TL.orgqr(f, m)
    opQ = Q.T if trans == "T" else Q
    CL = inputs.uniform_matrix(m, 7, 4)
    CR = inputs.uniform_matrix(5, m, 5)
    assert _rel(TL.ormqr(f, "L", trans, CL), opQ @ CL) <= 10 * m * U53
    assert _rel(TL.ormqr(f, "R", trans, CR), CR @ opQ) <= 10 * m * U53


@pytest.mark.parametrize("m,n,nb,ib,D", SHAPES[:3])
def test_ormqr_right_round_trip_and_transpose_identity(m, n, nb, ib, D):
    _, f = _factor(m, n, nb, ib, D, 6)
    C = inputs.normal_matrix(9, m, 7)
    back = TL.ormqr(f, "R", "T", TL.ormqr(f, "R", "N", C))
    assert _rel(back, C) <= 10 * m * U53
    # (C Q)^T = Q^T C^T: the right form against the left form
    assert _rel(TL.ormqr(f, "R", "N", C).T, TL.ormqr(f, "L", "T", C.T)) <= 4 * U53


def test_right_side_with_swapped_operator_is_caught():
    """A planted mistake (C Q computed as (Q C^T)^T) must fail the dense pin."""
    _, f = _factor(48, 32, 16, 4, 0, 8)
    C = inputs.normal_matrix(6, 48, 9)
    Q = TL.orgqr(f, 48)
    wrong = TL.apply_q(f, C.T).T
    assert _rel(wrong, C @ Q) > 1e-3
    assert _rel(TL.ormqr(f, "R", "N", C), C @ Q) <= 10 * 48 * U53


def test_empty_operands():
    _, f = _factor(40, 24, 16, 4, 0, 10)
    assert TL.orgqr(f, 0).shape == (40, 0)
    assert TL.ormqr(f, "R", "N", np.zeros((0, 40))).shape == (0, 40)
    assert TL.ormqr(f, "L", "T", np.zeros((40, 0))).shape == (40, 0)
