"""Pins for the tiled oracle (Section 3.1 kernels, Algorithm 1) against the
unblocked oracle (itself pinned), invariants and exact cases."""
import numpy as np
import pytest

from oracle import householder as H
from oracle import tiled as TL
from paper_0707_3548_gb300 import inputs
from tests._golden import exact_qr_cases

U53 = 2.0 ** -53


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


SHAPES = [
    # (m, n, nb, ib): full tiles, ragged tails, tall, wide, single tile
    (64, 64, 16, 4),
    (64, 64, 16, 16),
    (70, 45, 16, 8),
    (45, 70, 16, 4),
    (100, 30, 32, 8),
    (33, 33, 8, 2),
    (17, 5, 8, 8),
    (5, 17, 8, 4),
    (128, 96, 32, 32),
]


@pytest.mark.parametrize("m,n,nb,ib", SHAPES)
def test_tiled_r_equals_unblocked_r(m, n, nb, ib):
    A = inputs.uniform_matrix(m, n, 1000 + m + n + nb + ib)
    f = TL.tiled_qr(A, nb, ib)
    Ft, _ = H.geqr2(A)
    Rt = H.sign_normalize(f.R)
    Ru = H.sign_normalize(H.r_factor(Ft))
    k = min(m, n)
    assert _rel(Rt[:k], Ru[:k]) <= 1e-13
    assert np.array_equal(f.R, np.triu(f.R))


@pytest.mark.parametrize("m,n,nb,ib", SHAPES)
def test_tiled_invariants(m, n, nb, ib):
    A = inputs.normal_matrix(m, n, 7 + m * n + ib)
    f = TL.tiled_qr(A, nb, ib)
    Q = TL.form_q(f)
    R = f.R
    tol = 10 * max(m, n) * U53
    assert _rel(Q @ R, A) <= tol
    assert np.linalg.norm(np.eye(m) - Q.T @ Q) <= tol
    assert np.linalg.norm(R.T @ R - A.T @ A) / np.linalg.norm(A) ** 2 <= tol
    # apply_qt(A) = R and apply_q(apply_qt(B)) = B
    assert _rel(TL.apply_qt(f, A), R) <= tol
    B = inputs.normal_matrix(m, 3, 9)
    assert _rel(TL.apply_q(f, TL.apply_qt(f, B)), B) <= tol


def test_padding_rows_and_columns_stay_exactly_zero():
    m, n, nb, ib = 37, 29, 16, 4
    A = inputs.uniform_matrix(m, n, 3)
    f = TL.tiled_qr(A, nb, ib)
    assert not f.Ap[m:, :].any()          # padded rows stay zero (V and R)
    assert not np.triu(f.Ap)[:, n:].any()  # R is zero in padded columns


def test_padded_equals_unpadded_grid():
    """A 48 x 48 problem on a 16-grid equals the same problem embedded in
    padding (the pad only adds +0 terms)."""
    A = inputs.uniform_matrix(45, 45, 4)
    f1 = TL.tiled_qr(A, 16, 4)
    Ab = np.zeros((48, 48))
    Ab[:45, :45] = A
    f2 = TL.tiled_qr(Ab, 16, 4)
    assert np.allclose(f1.R, f2.R[:45, :45], rtol=0, atol=1e-14)


def test_ib_equals_nb_reproduces_unblocked_kernels():
    """With ib = b the tile kernels are the paper's unblocked DGEQT2/DTSQT2:
    GEQRT equals DGEQR2 + DLARFT on the tile, bit for bit."""
    nb = 12
    A = inputs.uniform_matrix(nb, nb, 5)
    F, T = TL.geqrt(A, nb)
    F2, tau = H.geqr2(A)
    T2 = H.larft(H.unit_lower(F2), tau)
    assert np.array_equal(F, F2)
    assert np.allclose(T, T2, rtol=0, atol=0)


def test_geqrt_blocked_equals_unblocked():
    nb = 32
    A = inputs.uniform_matrix(nb, nb, 6)
    for ib in (1, 2, 4, 8, 16, 32):
        F, T = TL.geqrt(A, ib)
        F2, tau = H.geqr2(A)
        assert _rel(F, F2) <= 1e-13
        # each T_l is DLARFT of its block's reflectors
        for l0 in range(0, nb, ib):
            V = H.unit_lower(F2[l0:, l0:l0 + ib], ib)
            assert np.allclose(T[:, l0:l0 + ib], H.larft(V, tau[l0:l0 + ib]), atol=1e-13)


@pytest.mark.parametrize("ib", [1, 4, 16])
def test_tsqrt_equals_qr_of_stacked_pair(ib):
    """DTSQT2 of [R; A] equals the unblocked QR of the stacked 2b x b matrix:
    same R (sign-normalised) and Q^T [R; A] = [R~; 0]."""
    nb = 16
    R0 = np.triu(inputs.uniform_matrix(nb, nb, 8))
    A0 = inputs.uniform_matrix(nb, nb, 9)
    lower = np.tril(inputs.uniform_matrix(nb, nb, 10), -1)  # V_kk stand-in
    R, V, T = TL.tsqrt(R0 + lower, A0, ib)
    assert np.array_equal(np.tril(R, -1), lower)               # lower part untouched
    S = np.vstack([R0, A0])
    F2, _ = H.geqr2(S)
    assert _rel(H.sign_normalize(np.triu(R)), H.sign_normalize(H.r_factor(F2)[:nb])) <= 1e-13
    # the stored reflectors reproduce the triangle: SSRFB applied to [R0; A0]
    top, bot = TL.ssrfb(R0, A0, V, T, ib, trans=True)
    assert _rel(top, np.triu(R)) <= 1e-13
    assert np.max(np.abs(bot)) <= 1e-13 * np.abs(R0).max()


@pytest.mark.parametrize("ib", [2, 8])
def test_ssrfb_and_larfb_are_orthogonal_and_inverse(ib):
    nb = 16
    A = inputs.uniform_matrix(2 * nb, nb, 12)
    f = TL.tiled_qr(A, nb, ib)
    X = inputs.normal_matrix(nb, 5, 13)
    Y = inputs.normal_matrix(nb, 5, 14)
    top, bot = TL.ssrfb(X, Y, f.tile(1, 0), f.T[(1, 0)], ib, trans=True)
    # norm preserved (orthogonal)
    assert abs(np.linalg.norm(np.vstack([top, bot])) - np.linalg.norm(np.vstack([X, Y]))) <= 1e-13 * np.linalg.norm(X)
    x2, y2 = TL.ssrfb(top, bot, f.tile(1, 0), f.T[(1, 0)], ib, trans=False)
    assert _rel(x2, X) <= 1e-14 and _rel(y2, Y) <= 1e-14
    Z = TL.larfb(X, f.tile(0, 0), f.T[(0, 0)], ib, trans=True)
    assert _rel(TL.larfb(Z, f.tile(0, 0), f.T[(0, 0)], ib, trans=False), X) <= 1e-14


@pytest.mark.parametrize("name,A,R", exact_qr_cases())
def test_tiled_exact_cases(name, A, R):
    for nb, ib in ((2, 1), (2, 2), (4, 2), (8, 4)):
        f = TL.tiled_qr(A, nb, ib)
        Rn = H.sign_normalize(f.R)[: R.shape[0]]
        assert np.allclose(Rn, R, rtol=0, atol=32 * U53 * np.abs(R).max())


def test_lapack_third_opinion_tiled():
    A = inputs.normal_matrix(96, 80, 77)
    f = TL.tiled_qr(A, 32, 8)
    Rl = H.sign_normalize(np.linalg.qr(A, mode="r"))
    assert _rel(H.sign_normalize(f.R)[:80], Rl[:80]) <= 1e-13
