"""Pins for the oracle's GMRES and GMRES-based refinement of the augmented
least-squares system (Carson, Higham and Pranesh 2020).

- GMRES (Saad and Schultz 1986): N steps on an N x N nonsingular system give
  its solution (the Krylov space is the whole space), compared with a dense
  solve; after k < N steps the residual is the minimum over the Krylov space,
  compared with a brute-force least-squares fit over the explicit Krylov
  vectors s, Ms, ..., M^{k-1} s.
- With the exact QR of A as preconditioner M equals the augmented matrix, so
  one GMRES step solves each correction equation.
- With the QR of A + E, ||E|| ~ 6e-8 ||A|| (an FP32 factorization's size of
  error) and kappa = 1e6 and 1e8, the refinement reaches backward error
  1e-14 and the exact least-squares solution of the stored A and b -- solved
  here in 60-digit decimal through the normal equations -- within the error
  bound of a backward-stable FP64 solver; at kappa = 1e8 the augmented-system
  refinement with the same factorization does not (kappa * 6e-8 = 6).
- Planted mistakes (an Arnoldi vector left unorthogonalised, the Hessenberg
  least-squares problem cut square, the correction subtracted, the residual
  without its -r term) must fail these pins."""
from decimal import Decimal, getcontext

import numpy as np
import pytest

from oracle import lstsq as L
from paper_0707_3548_gb300 import inputs

U64 = 2.0 ** -53


def _exact_ls_decimal(A, b, digits=60):
    """x with A^T A x = A^T b for the binary64 values of A and b, in decimal
    arithmetic of `digits` significant digits (Cholesky of A^T A, then two
    triangular solves).  kappa(A)^2 = 1e16 leaves about digits - 16 correct."""
    getcontext().prec = digits
    m, n = A.shape
    Ad = [[Decimal(float(A[i, j])) for j in range(n)] for i in range(m)]
    bd = [Decimal(float(v)) for v in b]
    G = [[sum(Ad[k][i] * Ad[k][j] for k in range(m)) for j in range(n)] for i in range(n)]
    c = [sum(Ad[k][i] * bd[k] for k in range(m)) for i in range(n)]
    Lc = [[Decimal(0)] * n for _ in range(n)]
    for j in range(n):
        s = G[j][j] - sum(Lc[j][k] * Lc[j][k] for k in range(j))
        Lc[j][j] = s.sqrt()
        for i in range(j + 1, n):
            Lc[i][j] = (G[i][j] - sum(Lc[i][k] * Lc[j][k] for k in range(j))) / Lc[j][j]
    y = [Decimal(0)] * n
    for i in range(n):
        y[i] = (c[i] - sum(Lc[i][k] * y[k] for k in range(i))) / Lc[i][i]
    x = [Decimal(0)] * n
    for i in reversed(range(n)):
        x[i] = (y[i] - sum(Lc[k][i] * x[k] for k in range(i + 1, n))) / Lc[i][i]
    return np.array([float(v) for v in x])


def _fp64_bound(A, b, x):
    """First-order forward-error bound of a backward-stable FP64 LS solver
    (perturbations of relative size u in A and b):
    u kappa (2 + (kappa + 1) ||r|| / (||A|| ||x||)), kappa = ||A|| ||A^+||."""
    s = np.linalg.svd(A, compute_uv=False)
    kappa = s[0] / s[-1]
    r = b - A @ x
    return U64 * kappa * (2.0 + (kappa + 1.0) * np.linalg.norm(r) / (s[0] * np.linalg.norm(x)))


def _problem(kappa, seed, m=60, n=20):
    A, b, _ = inputs.conditioned_ls_problem(m, n, kappa, seed=seed)
    E = 6e-8 * np.linalg.norm(A, 2) * inputs.normal_matrix(m, n, seed + 100) / np.sqrt(m)
    return A, b, L.QRSolver(A + E)


_EXACT = {}


def _exact(kappa, seed):
    if (kappa, seed) not in _EXACT:
        A, b, _ = _problem(kappa, seed)
        _EXACT[(kappa, seed)] = _exact_ls_decimal(A, b)
    return _EXACT[(kappa, seed)]


# ---- GMRES itself ----------------------------------------------------------------
def _gmres_pins_hold():
    N = 9
    M = inputs.normal_matrix(N, N, 31) + 3.0 * np.eye(N)
    s = inputs.normal_matrix(N, 1, 32)[:, 0]
    op = lambda z: M @ z  # noqa: E731
    z, steps, res = L.gmres(op, s, 0.0, N)
    if not (steps == N and np.linalg.norm(z - np.linalg.solve(M, s)) <= 1e-12 * np.linalg.norm(z)):
        return False
    for k in (1, 2, 3, 4):
        z, steps, res = L.gmres(op, s, 0.0, k)
        K = np.column_stack([np.linalg.matrix_power(M, i) @ s for i in range(k)])
        y = np.linalg.lstsq(M @ K, s, rcond=None)[0]
        best = np.linalg.norm(s - M @ (K @ y)) / np.linalg.norm(s)
        true = np.linalg.norm(s - M @ z) / np.linalg.norm(s)
        if not (steps == k and abs(true - best) <= 1e-10 and abs(res - true) <= 1e-10):
            return False
    return True


def test_gmres_finite_termination_and_krylov_minimum():
    assert _gmres_pins_hold()


def test_gmres_zero_right_hand_side():
    z, steps, res = L.gmres(lambda v: 2.0 * v, np.zeros(5), 1e-3, 10)
    assert steps == 0 and res == 0.0 and not np.any(z)


def test_gmres_breakdown_on_an_invariant_space_is_exact():
    # op = 2 I: K_1 is invariant, the first step is exact (h_21 = 0)
    s = np.arange(1.0, 6.0)
    z, steps, res = L.gmres(lambda v: 2.0 * v, s, 0.0, 5)
    assert steps == 1 and np.allclose(z, s / 2.0, rtol=0, atol=1e-15)


# ---- GMRES-IR ---------------------------------------------------------------------
def test_exact_preconditioner_solves_each_correction_in_one_step():
    A, b, _ = inputs.conditioned_ls_problem(50, 12, 1e3, seed=7)
    x0 = np.zeros(12)
    x, r, it, inner, hist = L.gmres_ir(A, b, L.QRSolver(A), tol=1e-15, inner_tol=1e-12, maxit=2, x0=x0)
    assert it >= 1 and inner <= 2 * it
    assert hist[1] <= 1e-15


def _ir_pins_hold(kappa, seed, solver_wrap=None):
    A, b, solver = _problem(kappa, seed)
    if solver_wrap is not None:
        solver = solver_wrap(solver)
    try:
        x, r, it, inner, hist = L.gmres_ir(A, b, solver, tol=1e-14, maxit=10)
    except (ValueError, np.linalg.LinAlgError, FloatingPointError):
        return False
    xe = _exact(kappa, seed)
    bound = _fp64_bound(A, b, xe)
    err = np.linalg.norm(x - xe) / np.linalg.norm(xe)
    return bool(hist[-1] <= 1e-14 and err <= 10.0 * bound and np.allclose(r, b - A @ x, rtol=0, atol=1e-8))


@pytest.mark.parametrize("kappa,seed", [(1e6, 1), (1e8, 1), (1e8, 2)])
def test_gmres_ir_reaches_the_exact_ls_solution(kappa, seed):
    assert _ir_pins_hold(kappa, seed)


def test_fp64_qr_solution_meets_the_same_bound():
    # the bound is attainable: the oracle's FP64 QR solve meets it too
    A, b, _ = _problem(1e8, 1)
    xe = _exact(1e8, 1)
    x = L.lstsq(A, b)
    assert np.linalg.norm(x - xe) / np.linalg.norm(xe) <= 10.0 * _fp64_bound(A, b, xe)


def test_augmented_refinement_fails_where_gmres_ir_succeeds():
    A, b, solver = _problem(1e8, 1)
    x, r, it, hist = L.augmented_refinement(A, b, solver, tol=1e-14, maxit=10)
    xe = _exact(1e8, 1)
    assert hist[-1] > 1e-12 or np.linalg.norm(x - xe) / np.linalg.norm(xe) > 10.0 * _fp64_bound(A, b, xe)


# ---- planted mistakes ------------------------------------------------------------
def _gmres_variant(skip_first=False, square=False):
    def gmres(op, s, tol, restart):
        beta = np.linalg.norm(s)
        if beta == 0.0:
            return np.zeros_like(s), 0, 0.0
        V = [s / beta]
        H = np.zeros((restart + 1, restart))
        for j in range(restart):
            w = op(V[j])
            for i in range(j + 1):
                if skip_first and i == 0 and j > 0:
                    continue
                H[i, j] = V[i] @ w
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            e1 = np.zeros(j + 2)
            e1[0] = beta
            if square:
                y = np.linalg.lstsq(H[:j + 1, :j + 1], e1[:j + 1], rcond=None)[0]
            else:
                y = np.linalg.lstsq(H[:j + 2, :j + 1], e1, rcond=None)[0]
            res = np.linalg.norm(e1 - H[:j + 2, :j + 1] @ y) / beta
            if res <= tol or H[j + 1, j] == 0.0 or j + 1 == restart:
                break
            V.append(w / H[j + 1, j])
        z = sum(y[i] * V[i] for i in range(j + 1))
        return z, j + 1, res
    return gmres


def test_unmutated_pins_hold():
    assert _gmres_pins_hold() and _ir_pins_hold(1e8, 1)


@pytest.mark.parametrize("variant", [dict(skip_first=True), dict(square=True)])
def test_mutated_gmres_fails_the_pins(monkeypatch, variant):
    monkeypatch.setattr(L, "gmres", _gmres_variant(**variant))
    assert not (_gmres_pins_hold() and _ir_pins_hold(1e8, 1))


def test_mutation_correction_subtracted(monkeypatch):
    orig = L.gmres

    def neg(op, s, tol, restart):
        z, steps, res = orig(op, s, tol, restart)
        return -z, steps, res
    monkeypatch.setattr(L, "gmres", neg)
    assert not _ir_pins_hold(1e8, 1)


def test_mutation_residual_without_r():
    # gmres_ir's outer step with f = b - A x in place of f = b - r - A x (the
    # preconditioner sees the wrong right-hand side), replayed step by step
    A, b, solver = _problem(1e8, 1)
    m, n = A.shape
    precond = L.augmented_preconditioner(solver)
    c = solver.qt(b[:, None])[:, 0]
    x = L.back_substitution(solver.R, c[:n])[:, 0]
    r = b - A @ x

    def op(z):
        u, v = precond(z[:m] + A @ z[m:], A.T @ z[:m])
        return np.concatenate([u, v])
    for _ in range(10):
        f = b - A @ x
        g = -(A.T @ r)
        u, v = precond(f, g)
        z, _, _ = L.gmres(op, np.concatenate([u, v]), 1e-3, 30)
        r, x = r + z[:m], x + z[m:]
    xe = _exact(1e8, 1)
    assert not (L.backward_error(A, x, b) <= 1e-14
                and np.linalg.norm(x - xe) / np.linalg.norm(xe) <= 10.0 * _fp64_bound(A, b, xe))


def test_gmres_ir_is_not_guaranteed_beyond_kappa_u_f_one():
    # kappa * 6e-8 = 6: on this seed the perturbed factor's smallest singular
    # values are ~5x those of A, the preconditioned matrix is ill conditioned
    # and the refinement stalls above the FP64 error bound -- the case the
    # library hands to an FP64 solve
    A, b, solver = _problem(1e8, 5)
    x, r, it, inner, hist = L.gmres_ir(A, b, solver, tol=1e-14, maxit=12)
    xe = _exact_ls_decimal(A, b)
    assert not (hist[-1] <= 1e-14 and np.linalg.norm(x - xe) / np.linalg.norm(xe) <= 10.0 * _fp64_bound(A, b, xe))
