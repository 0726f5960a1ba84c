"""Householder reflector, unblocked QR and the compact-WY T factor (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

Paper, Section 2 ("Block QR Factorization"): the QR factorization applies
min(m, n) Householder reflections; the panel is factored by DGEQR2 and the
reflectors are accumulated with DLARFT into an upper triangular T so that the
block reflector is applied by DLARFB (Eqs. lap_qr0-lap_qr2).  The paper takes
the reflector itself from the textbooks; this file uses the LAPACK convention
(reading recorded with the design notes):

    x = [alpha; x2],  ||x2|| == 0  ->  tau = 0, H = I, R_jj = alpha
    otherwise         beta = -sign(alpha) * ||x||   (sign(0) = +1)
                      tau  = (beta - alpha) / beta
                      v    = [1; x2 / (alpha - beta)],  R_jj = beta

so that H = I - tau v v^T maps x to [beta; 0].  Norms are scaled so entries
of magnitude up to 1e+-300 neither overflow nor underflow.

T convention (forward, columnwise; Schreiber and Van Loan, cited by the paper
for the compact WY form):  H_0 H_1 ... H_{k-1} = I - V T V^T with
    T[i, i] = tau_i,   T[0:i, i] = -tau_i * T[0:i, 0:i] @ (V[:, 0:i]^T v_i).
Q^T, the operator the factorization applies to A, is therefore I - V T^T V^T.
"""

import math

import numpy as np


def scaled_norm2(x):
    """Euclidean norm computed as s * sqrt(sum((x/s)^2)) with s = max|x_i|.

    The scaling keeps every square in [0, 1], so no intermediate overflows or
    underflows for finite inputs.  Inf and NaN propagate.
    """
    x = np.asarray(x, dtype=np.float64).ravel()
    if x.size == 0:
        return 0.0
    s = float(np.max(np.abs(x)))
    if s == 0.0 or not math.isfinite(s):
        return s
    y = x / s
    return s * math.sqrt(float(np.dot(y, y)))


def householder(alpha, x2):
    """Reflector annihilating x2 below alpha.

    Returns (tau, v2, beta) with H = I - tau [1; v2][1; v2]^T and
    H [alpha; x2] = [beta; 0].  Section 2 of the paper (DGEQR2 step).
    """
    alpha = float(alpha)
    x2 = np.asarray(x2, dtype=np.float64)
    xnorm = scaled_norm2(x2)
    if xnorm == 0.0:
        return 0.0, np.zeros_like(x2), alpha
    norm = math.hypot(alpha, xnorm)          # ||[alpha; x2]|| without overflow
    beta = -norm if alpha >= 0.0 else norm   # sign(0) = +1, also for -0.0
    tau = (beta - alpha) / beta
    v2 = x2 / (alpha - beta)
    return tau, v2, beta


def geqr2(A):
    """Unblocked Householder QR (DGEQR2), Section 2, Eq. lap_qr1.

    Returns (F, tau): F holds R on and above the diagonal and the reflectors'
    v (without their unit leading entry) below it; tau[j] is the scalar of
    reflector j.  Works for any m, n; min(m, n) reflectors.
    """
    F = np.array(A, dtype=np.float64, copy=True)
    m, n = F.shape
    kmax = min(m, n)
    tau = np.zeros(kmax)
    for j in range(kmax):
        t, v2, beta = householder(F[j, j], F[j + 1:, j])
        F[j, j] = beta
        F[j + 1:, j] = v2
        tau[j] = t
        if t != 0.0 and j + 1 < n:
            v = np.concatenate(([1.0], v2))
            w = v @ F[j:, j + 1:]                 # w = v^T A(j:, j+1:)
            F[j:, j + 1:] -= t * np.outer(v, w)   # A <- (I - tau v v^T) A
    return F, tau


def unit_lower(F, k=None):
    """Explicit V (m x k): the strictly lower part of F's first k columns with
    ones on the diagonal and zeros above it."""
    F = np.asarray(F, dtype=np.float64)
    m = F.shape[0]
    if k is None:
        k = min(F.shape)
    V = np.tril(F[:, :k], -1)
    for j in range(min(k, m)):
        V[j, j] = 1.0
    return V


def larft(V, tau):
    """Compact-WY T (DLARFT, forward direction, columnwise storage), Section 2.

    V is the explicit m x k matrix of reflector vectors; returns the k x k
    upper triangular T with H_0 H_1 ... H_{k-1} = I - V T V^T.
    """
    V = np.asarray(V, dtype=np.float64)
    k = len(tau)
    T = np.zeros((k, k))
    for i in range(k):
        T[i, i] = tau[i]
        if i > 0:
            T[:i, i] = -tau[i] * (T[:i, :i] @ (V[:, :i].T @ V[:, i]))
    return T


def reflector_product(V, tau):
    """H_0 H_1 ... H_{k-1} formed explicitly, one reflector at a time (used by
    the tests to pin the T convention by brute force)."""
    m = V.shape[0]
    H = np.eye(m)
    for i in range(len(tau)):
        v = V[:, i]
        H = H @ (np.eye(m) - tau[i] * np.outer(v, v))
    return H


def apply_qt(F, tau, B):
    """Q^T B from the unblocked factors, one reflector at a time in order."""
    C = np.array(B, dtype=np.float64, copy=True)
    m = F.shape[0]
    for j in range(len(tau)):
        if tau[j] == 0.0:
            continue
        v = np.concatenate(([1.0], F[j + 1:m, j]))
        w = v @ C[j:, :]
        C[j:, :] -= tau[j] * np.outer(v, w)
    return C


def apply_q(F, tau, B):
    """Q B from the unblocked factors: reflectors in reverse order."""
    C = np.array(B, dtype=np.float64, copy=True)
    m = F.shape[0]
    for j in reversed(range(len(tau))):
        if tau[j] == 0.0:
            continue
        v = np.concatenate(([1.0], F[j + 1:m, j]))
        w = v @ C[j:, :]
        C[j:, :] -= tau[j] * np.outer(v, w)
    return C


def form_q(F, tau):
    """Explicit m x m Q = H_0 H_1 ... H_{k-1}."""
    m = F.shape[0]
    return apply_q(F, tau, np.eye(m))


def r_factor(F):
    """The m x n upper trapezoidal R held on and above F's diagonal."""
    return np.triu(np.asarray(F, dtype=np.float64))


def sign_normalize(R):
    """D R with D = diag(sign(r_ii)), sign(0) = +1, so the diagonal is >= 0.

    For full-rank A this R is unique (it equals the Cholesky factor of A^T A),
    which lets factorizations computed in different orders be compared."""
    R = np.array(R, dtype=np.float64, copy=True)
    k = min(R.shape)
    for i in range(k):
        if R[i, i] < 0.0:
            R[i, :] = -R[i, :]
    return R
