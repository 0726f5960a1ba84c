"""Pins for the unblocked oracle (reflector, DGEQR2, DLARFT) against closed
forms, 50-digit brute force, LAPACK and invariants; none re-types the oracle."""
import math
from decimal import Decimal, getcontext

import numpy as np
import pytest

from oracle import householder as H
from paper_0707_3548_gb300 import inputs
from tests._golden import exact_qr_cases

U53 = 2.0 ** -53


# ---------------------------------------------------------------- reflector
def test_reflector_zero_tail_is_identity():
    tau, v2, beta = H.householder(-3.5, np.zeros(4))
    assert tau == 0.0 and beta == -3.5 and not v2.any()


def test_reflector_sign_of_zero_alpha_is_plus():
    # sign(0) = +1: beta = -||x||
    tau, v2, beta = H.householder(0.0, np.array([3.0, 4.0]))
    assert beta == -5.0 and tau == 1.0
    tau2, _, beta2 = H.householder(-0.0, np.array([3.0, 4.0]))
    assert beta2 == -5.0 and tau2 == 1.0


def test_reflector_maps_x_to_beta_e1():
    g = inputs.rng(3)
    for n in (1, 2, 7, 50):
        x = g.standard_normal(n + 1)
        tau, v2, beta = H.householder(x[0], x[1:])
        v = np.concatenate(([1.0], v2))
        Hx = x - tau * v * (v @ x)
        assert abs(Hx[0] - beta) <= 4 * U53 * abs(beta)
        assert np.max(np.abs(Hx[1:])) <= 8 * U53 * abs(beta)
        # H is orthogonal and symmetric: H^2 = I
        Hm = np.eye(n + 1) - tau * np.outer(v, v)
        assert np.allclose(Hm @ Hm, np.eye(n + 1), atol=1e-14)
        assert abs(abs(beta) - np.linalg.norm(x)) <= 4 * U53 * np.linalg.norm(x)


@pytest.mark.parametrize("scale", [1e300, 1e-300, 1e150, 1e-150])
def test_scaled_norm_no_overflow_underflow(scale):
    x = np.array([3.0, 4.0, 12.0]) * scale
    assert H.scaled_norm2(x) == pytest.approx(13.0 * scale, rel=4 * U53)
    tau, v2, beta = H.householder(x[0], x[1:])
    assert math.isfinite(tau) and np.all(np.isfinite(v2))
    assert abs(beta) == pytest.approx(13.0 * scale, rel=4 * U53)


# ---------------------------------------------------------------- closed forms
def test_2x2_closed_form():
    g = inputs.rng(11)
    for _ in range(200):
        a, b, c, d = g.uniform(-1, 1, 4)
        F, tau = H.geqr2(np.array([[a, b], [c, d]]))
        R = H.sign_normalize(H.r_factor(F))
        r11 = math.hypot(a, c)
        assert R[0, 0] == pytest.approx(r11, rel=4 * U53)
        assert R[0, 1] == pytest.approx((a * b + c * d) / r11, rel=1e-13, abs=1e-15)
        assert R[1, 1] == pytest.approx(abs(a * d - b * c) / r11, rel=1e-12, abs=1e-15)
        assert R[1, 0] == 0.0


@pytest.mark.parametrize("name,A,R", exact_qr_cases())
def test_exact_hand_built_cases(name, A, R):
    F, tau = H.geqr2(A)
    Rn = H.sign_normalize(H.r_factor(F))[: R.shape[0], :]
    assert np.allclose(Rn, R, rtol=0, atol=16 * U53 * np.abs(R).max())


# ---------------------------------------------------------------- brute force
def _dec(x):
    return Decimal(float(x))  # exact conversion of the binary64 value


def _cholesky_r_decimal(A):
    """Positive-diagonal R with R^T R = A^T A, in 50-digit decimal."""
    getcontext().prec = 50
    m, n = A.shape
    G = [[sum(_dec(A[r, i]) * _dec(A[r, j]) for r in range(m)) for j in range(n)] for i in range(n)]
    R = [[Decimal(0)] * n for _ in range(n)]
    for i in range(n):
        s = G[i][i] - sum(R[k][i] * R[k][i] for k in range(i))
        R[i][i] = s.sqrt()
        for j in range(i + 1, n):
            R[i][j] = (G[i][j] - sum(R[k][i] * R[k][j] for k in range(i))) / R[i][i]
    return np.array([[float(v) for v in row] for row in R])


def _gram_schmidt_r_decimal(A):
    """Classical Gram-Schmidt R (r_ij = q_i^T a_j) in 50-digit decimal."""
    getcontext().prec = 50
    m, n = A.shape
    cols = [[_dec(A[r, j]) for r in range(m)] for j in range(n)]
    Q = []
    R = [[Decimal(0)] * n for _ in range(n)]
    for j in range(n):
        v = list(cols[j])
        for i, qi in enumerate(Q):
            R[i][j] = sum(a * b for a, b in zip(qi, cols[j]))
            v = [vv - R[i][j] * qq for vv, qq in zip(v, qi)]
        R[j][j] = sum(vv * vv for vv in v).sqrt()
        Q.append([vv / R[j][j] for vv in v])
    return np.array([[float(v) for v in row] for row in R])


@pytest.mark.parametrize("m,n,seed", [(1, 1, 0), (2, 2, 1), (3, 2, 2), (4, 4, 3), (6, 6, 4), (6, 3, 5), (5, 5, 6)])
def test_brute_force_decimal(m, n, seed):
    A = inputs.uniform_matrix(m, n, seed)
    F, tau = H.geqr2(A)
    R = H.sign_normalize(H.r_factor(F))[:n, :]
    Rc = _cholesky_r_decimal(A)
    Rg = _gram_schmidt_r_decimal(A)
    assert np.allclose(Rc, Rg, rtol=0, atol=1e-30 + 1e-25)  # the two brute forces agree
    scale = np.abs(Rc).max()
    kappa = np.linalg.cond(A)
    assert np.max(np.abs(R - Rc)) <= 50 * n * U53 * kappa * scale


# ---------------------------------------------------------------- invariants
@pytest.mark.parametrize("m,n", [(64, 64), (100, 37), (37, 100), (256, 256), (300, 1)])
def test_invariants_qr(m, n):
    A = inputs.uniform_matrix(m, n, m * 7 + n)
    F, tau = H.geqr2(A)
    R = H.r_factor(F)
    Q = H.form_q(F, tau)
    k = max(m, n)
    tol = 10 * k * U53
    assert np.linalg.norm(A - Q @ R) / np.linalg.norm(A) <= tol
    assert np.linalg.norm(np.eye(m) - Q.T @ Q) <= tol
    assert np.array_equal(R, np.triu(R))               # strictly upper
    assert np.linalg.norm(R.T @ R - A.T @ A) / np.linalg.norm(A) ** 2 <= tol
    # Q^T A = R through the apply path as well
    assert np.linalg.norm(H.apply_qt(F, tau, A) - R) / np.linalg.norm(A) <= tol


@pytest.mark.parametrize("m,n", [(50, 50), (90, 40), (40, 90)])
def test_lapack_third_opinion(m, n):
    A = inputs.normal_matrix(m, n, 42)
    F, tau = H.geqr2(A)
    R = H.sign_normalize(H.r_factor(F))
    Rl = H.sign_normalize(np.linalg.qr(A, mode="r"))
    k = min(m, n)
    assert np.allclose(R[:k], Rl[:k], rtol=0, atol=1e-12 * np.abs(Rl).max())


@pytest.mark.parametrize("m,k", [(12, 5), (30, 30), (9, 1)])
def test_larft_equals_reflector_product(m, k):
    """H_0 H_1 ... H_{k-1} built one reflector at a time equals I - V T V^T."""
    A = inputs.normal_matrix(m, k, 5)
    F, tau = H.geqr2(A)
    V = H.unit_lower(F, k)
    T = H.larft(V, tau)
    assert np.array_equal(T, np.triu(T))
    P = H.reflector_product(V, tau)
    assert np.allclose(P, np.eye(m) - V @ T @ V.T, atol=1e-13)
    # and the factorization applies the transpose: (I - V T^T V^T) A = R
    R = H.r_factor(F)
    assert np.allclose((np.eye(m) - V @ T.T @ V.T) @ A, R, atol=1e-12)


def test_rank_deficient_column_gets_tau_zero():
    A = inputs.normal_matrix(6, 3, 1)
    A[:, 1] = 0.0
    F, tau = H.geqr2(A)
    assert tau[1] == 0.0 and F[1, 1] == 0.0
