"""Least squares through the QR factors, its backward error, and
augmented-system iterative refinement (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``).

The paper names applying Q and forming Q as the natural follow-ups of the
tiled factorization (Section 5); least squares is their first user:
    min ||A x - b||,  A = Q [R; 0]  =>  x = R[:n, :n]^{-1} (Q^T b)[:n].

Backward error (the paper is silent; normwise reading recorded with the
design notes):
    eta(x) = ||A^T r||_2 / (||A||_F (||A||_F ||x||_2 + ||b||_2)),  r = b - A x.

Refinement (the paper is silent), three forms:

(1) corrected semi-normal equations (Bjorck): with R from a (possibly lower
accuracy) QR factorization, R^T R ~ A^T A, and float64 residuals
    e = b - A x,  dx = R^{-1} (R^{-T} (A^T e)),  x += dx.
Its fixed point is the LS solution (A^T (b - A x) = 0).  When R is the
exact factor of A + E with ||E|| = eps ||A||, the iteration matrix
I - (R^T R)^{-1} A^T A is similar to I - M^T M, M = A R^{-1} = Q - E R^{-1},
so the error contracts by about 2 kappa(A) eps per step: it needs
kappa eps well below 1;

(2) Bjorck's iterative refinement of the augmented system
    [ I   A ] [r]   [b]
    [ A^T 0 ] [x] = [0]
with residuals in float64 and each correction solved through a QR
factorization (possibly of lower accuracy):
    f = b - r - A x,  g = -A^T r
    h  = R^{-T} g,  d = Q^T f = [d1; d2]
    dx = R^{-1} (d1 - h),  dr = Q [h; d2]
    x += dx, r += dr.

(3) GMRES-based refinement of the same augmented system (Carson, Higham and
Pranesh, "Three-precision GMRES-based iterative refinement for least squares
problems", SIAM J. Sci. Comput. 2020), for problems too ill-conditioned for
(2) to contract: each outer step solves the correction equation
    [I A; A^T 0] [dr; dx] = [f; g]
by GMRES (Saad and Schultz 1986) applied to the left-preconditioned system
M^{-1} [I A; A^T 0] z = M^{-1} [f; g], where M is the augmented matrix with
the factorization's Q R in place of A, so that M^{-1} [f; g] is exactly the
correction of (2).  The preconditioned matrix stays well conditioned when
kappa(A) u_f is near or above 1, where (2) stalls.  Readings (the method's
paper leaves them to the user): the augmented system is not scaled
(alpha = 1, as in (2)); the inner solve stops at a relative residual
inner_tol or after `restart` steps, and the outer step applies whatever it
reached.
"""

import numpy as np

from .householder import geqr2, apply_qt as _apply_qt_unblocked, apply_q as _apply_q_unblocked


def back_substitution(R, C):
    """Solve R X = C for upper triangular n x n R, one row at a time from the
    bottom (plain loop)."""
    R = np.asarray(R, dtype=np.float64)
    X = np.array(C, dtype=np.float64, copy=True)
    if X.ndim == 1:
        X = X[:, None]
    n = R.shape[0]
    for i in reversed(range(n)):
        if i + 1 < n:
            X[i, :] -= R[i, i + 1:n] @ X[i + 1:n, :]
        X[i, :] /= R[i, i]
    return X


def forward_substitution_rt(R, G):
    """Solve R^T H = G for upper triangular R (so R^T is lower), top down."""
    R = np.asarray(R, dtype=np.float64)
    H = np.array(G, dtype=np.float64, copy=True)
    if H.ndim == 1:
        H = H[:, None]
    n = R.shape[0]
    for i in range(n):
        if i > 0:
            H[i, :] -= R[:i, i] @ H[:i, :]
        H[i, :] /= R[i, i]
    return H


class QRSolver:
    """Least-squares solves from one unblocked QR factorization (m >= n)."""

    def __init__(self, A):
        A = np.asarray(A, dtype=np.float64)
        self.m, self.n = A.shape
        assert self.m >= self.n
        self.F, self.tau = geqr2(A)
        self.R = np.triu(self.F[:self.n, :self.n])

    def qt(self, B):
        return _apply_qt_unblocked(self.F, self.tau, B)

    def q(self, B):
        return _apply_q_unblocked(self.F, self.tau, B)

    def solve(self, B):
        B = np.asarray(B, dtype=np.float64)
        vec = B.ndim == 1
        C = self.qt(B[:, None] if vec else B)
        X = back_substitution(self.R, C[:self.n])
        return X[:, 0] if vec else X


def lstsq(A, B):
    """x = argmin ||A x - b|| for full-rank m x n A, m >= n."""
    return QRSolver(A).solve(B)


def backward_error(A, x, b):
    """Normwise backward error of an LS solution (columnwise for several
    right-hand sides: returns the max over columns)."""
    A = np.asarray(A, dtype=np.float64)
    x = np.asarray(x, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    if x.ndim == 1:
        x = x[:, None]
        b = b[:, None]
    nA = np.linalg.norm(A, "fro")
    worst = 0.0
    for c in range(x.shape[1]):
        r = b[:, c] - A @ x[:, c]
        eta = np.linalg.norm(A.T @ r) / (nA * (nA * np.linalg.norm(x[:, c]) + np.linalg.norm(b[:, c])))
        worst = max(worst, eta)
    return worst


def augmented_refinement(A, b, solver, tol=1e-12, maxit=30, x0=None):
    """Bjorck's refinement of the augmented system with float64 residuals.

    ``solver`` is a QRSolver-like object (methods qt, q and attribute R) of a
    possibly perturbed or lower-accuracy factorization of A.  Returns
    (x, r, iterations, backward errors per iteration).
    """
    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64).ravel()
    m, n = A.shape
    R = np.asarray(solver.R, dtype=np.float64)
    if x0 is None:
        c = np.asarray(solver.qt(b[:, None]), dtype=np.float64)[:, 0]
        x = back_substitution(R, c[:n])[:, 0]
    else:
        x = np.array(x0, dtype=np.float64)
    r = b - A @ x
    history = [backward_error(A, x, b)]
    it = 0
    while history[-1] > tol and it < maxit:
        f = b - r - A @ x
        g = -(A.T @ r)
        h = forward_substitution_rt(R, g)[:, 0]
        d = np.asarray(solver.qt(f[:, None]), dtype=np.float64)[:, 0]
        dx = back_substitution(R, (d[:n] - h)[:, None])[:, 0]
        y = np.concatenate([h, d[n:]])
        dr = np.asarray(solver.q(y[:, None]), dtype=np.float64)[:, 0]
        x = x + dx
        r = r + dr
        it += 1
        history.append(backward_error(A, x, b))
    return x, r, it, history


def seminormal_refinement(A, b, R, tol=1e-12, maxit=30, x0=None):
    """Corrected semi-normal equations with float64 residuals:
    x += R^{-1} R^{-T} A^T (b - A x) until the backward error is at most tol.

    ``R`` is the n x n upper triangle of a possibly lower-accuracy QR
    factorization of A.  Starts from x0 (default: the semi-normal solution
    R^{-1} R^{-T} A^T b).  Returns (x, iterations, backward errors per
    iteration).
    """
    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64).ravel()
    R = np.asarray(R, dtype=np.float64)

    def correction(v):
        return back_substitution(R, forward_substitution_rt(R, (A.T @ v)[:, None]))[:, 0]

    x = correction(b) if x0 is None else np.array(x0, dtype=np.float64)
    history = [backward_error(A, x, b)]
    it = 0
    while history[-1] > tol and it < maxit:
        x = x + correction(b - A @ x)
        it += 1
        history.append(backward_error(A, x, b))
    return x, it, history


def gmres(op, s, tol, restart):
    """GMRES for op(z) = s from z = 0 (Saad and Schultz 1986).

    Arnoldi with modified Gram-Schmidt builds an orthonormal basis V_k of the
    Krylov space K_k(op, s) and the (k+1) x k Hessenberg H_k with
    op(V_k) = V_{k+1} H_k; the iterate z_k = V_k y_k takes the y_k that
    minimises ||beta e_1 - H_k y|| (beta = ||s||), which minimises the
    residual ||s - op(z)|| over the Krylov space.  Stops once that residual is
    at most tol * beta, at a breakdown (h_{k+1,k} = 0: the space is invariant
    and z_k solves the system), or after `restart` steps.

    Returns (z, steps, relative residual)."""
    s = np.asarray(s, dtype=np.float64)
    beta = np.linalg.norm(s)
    if beta == 0.0:
        return np.zeros_like(s), 0, 0.0
    V = [s / beta]
    H = np.zeros((restart + 1, restart))
    for j in range(restart):
        w = np.asarray(op(V[j]), dtype=np.float64)
        for i in range(j + 1):
            H[i, j] = V[i] @ w
            w = w - H[i, j] * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        e1 = np.zeros(j + 2)
        e1[0] = beta
        y = np.linalg.lstsq(H[:j + 2, :j + 1], e1, rcond=None)[0]
        res = np.linalg.norm(e1 - H[:j + 2, :j + 1] @ y) / beta
        if res <= tol or H[j + 1, j] == 0.0 or j + 1 == restart:
            break
        V.append(w / H[j + 1, j])
    z = np.zeros_like(s)
    for i in range(j + 1):
        z = z + y[i] * V[i]
    return z, j + 1, res


def augmented_preconditioner(solver):
    """M^{-1} for the augmented system [I A; A^T 0] with A replaced by the
    factorization Q R of ``solver`` (methods qt, q and attribute R):
    M^{-1} [f; g] = [Q [h; d2]; R^{-1} (d1 - h)],  h = R^{-T} g,  d = Q^T f
    (the correction of Bjorck's refinement, form (2))."""
    R = np.asarray(solver.R, dtype=np.float64)
    n = R.shape[0]

    def apply(f, g):
        h = forward_substitution_rt(R, np.asarray(g, dtype=np.float64)[:, None])[:, 0]
        d = np.asarray(solver.qt(np.asarray(f, dtype=np.float64)[:, None]), dtype=np.float64)[:, 0]
        v = back_substitution(R, (d[:n] - h)[:, None])[:, 0]
        u = np.asarray(solver.q(np.concatenate([h, d[n:]])[:, None]), dtype=np.float64)[:, 0]
        return u, v

    return apply


def gmres_ir(A, b, solver, tol=1e-12, inner_tol=1e-3, restart=30, maxit=20, x0=None, settle=True):
    """GMRES-based iterative refinement of the augmented system, left-
    preconditioned by the factorization in ``solver`` (form (3) above).

    Starts from x0 (default: the solution through the factorization) and
    r = b - A x; each outer step forms in float64
        f = b - r - A x,  g = -A^T r,
    solves [I A; A^T 0] [dr; dx] = [f; g] by GMRES on the left-preconditioned
    system to a relative residual inner_tol (at most `restart` steps), and
    updates r += dr, x += dx, until the backward error is at most tol and,
    with ``settle``, x has settled: the last correction is below FP64
    rounding (||dx|| <= 2^-50 ||x||) or no longer halves the one before (the
    corrections have reached the rounding noise of the float64 residuals).
    A backward error at tol alone does not make x accurate when kappa(A) is
    large; the settled x is as accurate as a backward-stable FP64 solve.
    Stops after maxit outer steps in any case.

    Returns (x, r, outer steps, total GMRES steps, backward errors per outer
    step)."""
    A = np.asarray(A, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64).ravel()
    m, n = A.shape
    precond = augmented_preconditioner(solver)
    if x0 is None:
        c = np.asarray(solver.qt(b[:, None]), dtype=np.float64)[:, 0]
        x = back_substitution(np.asarray(solver.R, dtype=np.float64), c[:n])[:, 0]
    else:
        x = np.array(x0, dtype=np.float64)
    r = b - A @ x

    def op(z):
        u, v = precond(z[:m] + A @ z[m:], A.T @ z[:m])
        return np.concatenate([u, v])

    history = [backward_error(A, x, b)]
    it = 0
    inner = 0
    dx_prev = np.inf
    settled = not settle
    while (history[-1] > tol or not settled) and it < maxit:
        f = b - r - A @ x
        g = -(A.T @ r)
        u, v = precond(f, g)
        z, steps, _ = gmres(op, np.concatenate([u, v]), inner_tol, restart)
        inner += steps
        r = r + z[:m]
        x = x + z[m:]
        it += 1
        history.append(backward_error(A, x, b))
        dx = np.linalg.norm(z[m:])
        settled = (not settle) or dx <= 2.0 ** -50 * np.linalg.norm(x) or not (dx < 0.5 * dx_prev)
        dx_prev = min(dx_prev, dx)
    return x, r, it, inner, history
