"""Pins for the least-squares oracle and Bjorck's refinement."""
import numpy as np
import pytest

from oracle import householder as H
from oracle import lstsq as L
from oracle import tiled as TL
from paper_0707_3548_gb300 import inputs


def test_triangular_solves_against_scipy():
    import scipy.linalg as sla
    R = np.triu(inputs.uniform_matrix(20, 20, 1)) + 5 * np.eye(20)
    C = inputs.normal_matrix(20, 3, 2)
    assert np.allclose(L.back_substitution(R, C), sla.solve_triangular(R, C), atol=1e-13)
    assert np.allclose(L.forward_substitution_rt(R, C), sla.solve_triangular(R, C, trans="T"), atol=1e-13)


@pytest.mark.parametrize("m,n", [(60, 20), (200, 50), (30, 30)])
def test_lstsq_normal_equations_and_lapack(m, n):
    A = inputs.normal_matrix(m, n, 3)
    b = inputs.normal_matrix(m, 2, 4)
    x = L.lstsq(A, b)
    r = b - A @ x
    # A^T r = 0 (normal equations), relative to ||A|| (||A|| ||x|| + ||b||)
    nA = np.linalg.norm(A)
    assert np.linalg.norm(A.T @ r) <= 1e-13 * nA * (nA * np.linalg.norm(x) + np.linalg.norm(b))
    xl = np.linalg.lstsq(A, b, rcond=None)[0]
    assert np.allclose(x, xl, atol=1e-12)
    assert L.backward_error(A, x, b) <= 1e-15


def test_backward_error_zero_for_exact_solution_and_positive_otherwise():
    A = inputs.normal_matrix(40, 10, 5)
    x = inputs.normal_matrix(10, 1, 6)[:, 0]
    b = A @ x
    assert L.backward_error(A, x, b) <= 1e-15
    assert L.backward_error(A, x + 1e-3, b) > 1e-6


def test_tiled_lstsq_equals_unblocked():
    A = inputs.normal_matrix(90, 40, 7)
    b = inputs.normal_matrix(90, 1, 8)
    f = TL.tiled_qr(A, 16, 4)
    c = TL.apply_qt(f, b)
    x = L.back_substitution(f.R[:40, :40], c[:40])
    assert np.allclose(x, L.lstsq(A, b), atol=1e-12)


class _PerturbedSolver(L.QRSolver):
    """QR of A + E: a stand-in for a lower-accuracy factorization."""


@pytest.mark.parametrize("kappa", [1e2, 1e5])
def test_augmented_refinement_converges_to_exact_ls(kappa):
    A, b, _ = inputs.conditioned_ls_problem(300, 40, kappa, seed=1)
    x_ref = L.lstsq(A, b)
    E = 1e-7 * np.linalg.norm(A, 2) * inputs.normal_matrix(300, 40, 9) / np.sqrt(300)
    solver = _PerturbedSolver(A + E)
    x, r, it, hist = L.augmented_refinement(A, b, solver, tol=1e-14, maxit=50)
    assert hist[-1] <= 1e-14
    assert hist[0] > hist[-1]
    assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) <= 1e-12 * kappa
    assert np.allclose(r, b - A @ x, atol=1e-10)


def test_conditioned_problem_has_requested_condition_number():
    for kappa in (1e2, 1e5, 1e8):
        A, b, x = inputs.conditioned_ls_problem(200, 30, kappa, seed=2)
        s = np.linalg.svd(A, compute_uv=False)
        assert s[0] / s[-1] == pytest.approx(kappa, rel=1e-3 if kappa < 1e8 else 1e-1)


def test_seminormal_refinement_with_exact_r_is_the_ls_solution():
    """With the exact R, R^T R = A^T A, so the first semi-normal solve is the
    normal-equations solution: one correction reaches the FP64 LS answer."""
    A, b, _ = inputs.conditioned_ls_problem(200, 30, 1e3, seed=4)
    R = np.linalg.qr(A, mode="r")
    x, it, hist = L.seminormal_refinement(A, b, R, tol=1e-15, maxit=3)
    x_ref = np.linalg.lstsq(A, b, rcond=None)[0]
    assert it <= 2 and hist[-1] <= 1e-15
    assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) <= 1e-14 * 1e3


@pytest.mark.parametrize("kappa", [1e1, 1e2])
def test_seminormal_refinement_converges_for_well_conditioned_problems(kappa):
    """An R perturbed by eps ~ 1e-7 relative (an FP32 factorization's size of
    error) contracts the error by ~ 2 kappa eps per step."""
    A, b, _ = inputs.conditioned_ls_problem(300, 40, kappa, seed=1)
    E = 1e-7 * np.linalg.norm(A, 2) * inputs.normal_matrix(300, 40, 9) / np.sqrt(300)
    R = _PerturbedSolver(A + E).R
    x, it, hist = L.seminormal_refinement(A, b, R, tol=1e-14, maxit=20)
    assert hist[-1] <= 1e-14 and it <= 6
    x_ref = L.lstsq(A, b)
    assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) <= 1e-12 * kappa
    # geometric decrease while far from rounding level
    for a, c in zip(hist[:-1], hist[1:]):
        if c > 1e-15:
            assert c < 0.1 * a


def test_seminormal_refinement_diverges_when_kappa_eps_exceeds_one():
    """R is the exact factor of A + E, so R^T R = (A+E)^T (A+E) and the
    iteration matrix is similar to M^T M - I with M = A R^-1 = Q - E R^-1:
    the contraction is about 2 kappa eps.  kappa eps = 1e5 * 1e-3 = 100: the
    corrections grow (the regime the device leaves for the augmented-system
    refinement)."""
    A, b, _ = inputs.conditioned_ls_problem(300, 40, 1e5, seed=1)
    E = 1e-3 * np.linalg.norm(A, 2) * inputs.normal_matrix(300, 40, 9) / np.sqrt(300)
    R = _PerturbedSolver(A + E).R
    x_ref = L.lstsq(A, b)
    x, it, hist = L.seminormal_refinement(A, b, R, tol=0.0, maxit=4)
    assert np.linalg.norm(x - x_ref) > np.linalg.norm(x_ref)
