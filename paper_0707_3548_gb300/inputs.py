"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle
checks.

This module only draws numbers (NumPy PCG64, seeded) and arranges them; it
holds none of the QR method's arithmetic.  The one non-trivial recipe, the
random orthonormal factors of the conditioned least-squares problems, uses
two passes of Cholesky orthonormalisation (Gram matrix + Cholesky + a
triangular solve), not a Householder QR.

All matrices come back in column-major (Fortran) order, so their buffers can
be handed to the C ABI with leading dimension m.
"""

import math

import numpy as np


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def uniform_matrix(m, n, seed, lo=-1.0, hi=1.0):
    """m x n, entries iid uniform[lo, hi)."""
    return np.asfortranarray(rng(seed).uniform(lo, hi, size=(m, n)))


def normal_matrix(m, n, seed):
    """m x n, entries iid N(0, 1)."""
    return np.asfortranarray(rng(seed).standard_normal(size=(m, n)))


def _orthonormal_columns(G):
    """Orthonormalise the columns of a full-rank Gaussian G (m >= n) by two
    passes of Cholesky orthonormalisation: Y <- Y C^{-1}, C^T C = Y^T Y.
    The positive-diagonal triangular factor is unique, so in exact arithmetic
    this is the Haar-distributed orthonormal factor of G."""
    import scipy.linalg as sla

    Y = np.array(G, dtype=np.float64)
    for _ in range(2):
        C = np.linalg.cholesky(Y.T @ Y).T               # upper, C^T C = Y^T Y
        Y = sla.solve_triangular(C, Y.T, trans="T", lower=False).T
    return Y


def conditioned_ls_problem(m, n, kappa, seed, noise=1e-6):
    """Least-squares test problem A = U diag(sigma) V^T with U (m x n) and V
    (n x n) orthonormal, sigma_i = kappa^(-i/(n-1)) (i = 0..n-1, geometric),
    x_true ~ N(0, 1), b = A x_true + noise * N(0, 1).

    Returns (A, b, x_true), A column-major."""
    g = rng(seed)
    U = _orthonormal_columns(g.standard_normal(size=(m, n)))
    V = _orthonormal_columns(g.standard_normal(size=(n, n)))
    if n > 1:
        sigma = kappa ** (-np.arange(n) / (n - 1.0))
    else:
        sigma = np.ones(1)
    A = np.asfortranarray((U * sigma) @ V.T)
    x_true = g.standard_normal(n)
    b = A @ x_true + noise * g.standard_normal(m)
    return A, b, x_true


def batch_shapes(count, seed, m_lo=64, m_hi=2048, n_lo=32):
    """Shapes of a batch of independent problems: m = round(exp(U[ln m_lo,
    ln m_hi])), n uniform on {n_lo, ..., m}."""
    g = rng(seed)
    ms = np.rint(np.exp(g.uniform(math.log(m_lo), math.log(m_hi), size=count))).astype(int)
    ms = np.clip(ms, m_lo, m_hi)
    ns = np.array([g.integers(min(n_lo, m), m + 1) for m in ms], dtype=int)
    return list(zip(ms.tolist(), ns.tolist()))


def batch_matrices(shapes, seed):
    """One N(0,1) matrix per shape, each from its own derived seed."""
    return [normal_matrix(m, n, seed * 1_000_003 + t) for t, (m, n) in enumerate(shapes)]


def serving_stream(rate, window_s, seed, m_lo=128, m_hi=8192, n_lo=64,
                   nrhs_hi=16, repeat_frac=0.3, fp32_frac=0.5):
    """Poisson request stream for the least-squares server.

    Each request: arrival time (s), m log-uniform in [m_lo, m_hi], n uniform
    in [n_lo, max(n_lo, m // 2)], nrhs uniform on {1..nrhs_hi}, a matrix id
    (a repeat request reuses an earlier id, i.e. the same A), and a precision
    class ("fp64" or "fp32r").  Matrices are not materialised here."""
    g = rng(seed)
    t = 0.0
    reqs = []
    mats = []
    while True:
        t += g.exponential(1.0 / rate)
        if t >= window_s:
            break
        if mats and g.uniform() < repeat_frac:
            mid = int(g.integers(0, len(mats)))
        else:
            m = int(round(math.exp(g.uniform(math.log(m_lo), math.log(m_hi)))))
            m = min(max(m, m_lo), m_hi)
            n = int(g.integers(min(n_lo, m), max(n_lo, m // 2) + 1))
            n = min(n, m)
            mats.append((m, n, len(mats)))
            mid = len(mats) - 1
        nrhs = int(g.integers(1, nrhs_hi + 1))
        cls = "fp32r" if g.uniform() < fp32_frac else "fp64"
        reqs.append({"t": t, "matrix": mid, "m": mats[mid][0], "n": mats[mid][1],
                     "nrhs": nrhs, "prec": cls})
    return reqs, mats
