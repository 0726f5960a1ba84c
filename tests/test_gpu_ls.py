"""GPU least squares (tqr_solve_ls) against the oracle."""
import numpy as np
import pytest

from oracle import lstsq as LS
from paper_0707_3548_gb300 import inputs, tqr
from tests.gpu_util import to_dev, to_host, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("m,n,nrhs,nb,ib", [(700, 300, 1, 128, 32), (500, 500, 3, 64, 16), (1000, 130, 17, 64, 32)])
def test_solve_fp64_matches_oracle(m, n, nrhs, nb, ib):
    torch_cuda()
    A = inputs.normal_matrix(m, n, 31)
    B = inputs.normal_matrix(m, nrhs, 32)
    X, it, berr, rc = tqr.tqr_solve_ls(to_dev(A), to_dev(B), nb=nb, ib=ib)
    assert rc == tqr.TQR_OK and it == 0
    Xo = LS.lstsq(A, B)
    assert np.max(np.abs(to_host(X) - Xo)) <= 1e-10 * max(1.0, np.abs(Xo).max())
    assert berr <= 1e-14
    assert abs(berr - LS.backward_error(A, to_host(X), B)) <= 1e-15 + 0.05 * berr


def test_reported_backward_error_is_the_oracles():
    """Without refinement (maxit = 0) the FP32 solution's backward error is
    well above rounding noise, so the device's value (FP64 residual, ||A||_F,
    ||x||, ||b||) must equal the oracle's for the returned x closely."""
    torch_cuda()
    A, b, _ = inputs.conditioned_ls_problem(1500, 400, 1e3, seed=2)
    X, it, berr, rc = tqr.tqr_solve_ls(to_dev(A), to_dev(b[:, None]), prec=tqr.TQR_PREC_FP32, tol=1e-12,
                                       maxit=0, nb=64, ib=16, check=False)
    assert rc == tqr.TQR_ERR_NOCONV and it == 0
    ref = LS.backward_error(A, to_host(X)[:, 0], b)
    assert ref > 1e-12
    assert abs(berr - ref) <= 1e-6 * ref


def test_nonfinite_input_is_reported():
    torch_cuda()
    A = inputs.normal_matrix(200, 60, 7)
    B = inputs.normal_matrix(200, 2, 8)
    A_nan = A.copy()
    A_nan[17, 5] = np.nan
    _, _, _, rc = tqr.tqr_solve_ls(to_dev(A_nan), to_dev(B), nb=32, ib=8, check=False)
    assert rc == tqr.TQR_ERR_NONFINITE
    B_inf = B.copy()
    B_inf[3, 1] = np.inf
    _, _, _, rc = tqr.tqr_solve_ls(to_dev(A), to_dev(B_inf), prec=tqr.TQR_PREC_FP32, nb=32, ib=8, check=False)
    assert rc == tqr.TQR_ERR_NONFINITE


@pytest.mark.parametrize("kappa", [1e2, 1e5])
def test_solve_fp32_refined_reaches_fp64_accuracy(kappa):
    torch_cuda()
    A, b, _ = inputs.conditioned_ls_problem(2000, 500, kappa, seed=1)
    X, it, berr, rc = tqr.tqr_solve_ls(to_dev(A), to_dev(b[:, None]), prec=tqr.TQR_PREC_FP32, tol=1e-12,
                                       maxit=30, nb=64, ib=16)
    assert rc == tqr.TQR_OK, (rc, it, berr)
    assert berr <= 1e-12 and it >= 1
    xo = LS.lstsq(A, b)
    assert np.linalg.norm(to_host(X)[:, 0] - xo) / np.linalg.norm(xo) <= 1e-13 * kappa
    assert LS.backward_error(A, to_host(X)[:, 0], b) <= 1e-12



@pytest.mark.parametrize("case", ["dominant_top", "graded_columns", "gaussian"])
def test_fp32_factor_is_accurate_at_fp32_level(case):
    """The FP32 factorization alone (no refinement) must solve to a backward
    error of a modest multiple of the FP32 unit roundoff, also where the
    panel's running column sums cancel heavily: a matrix whose top block
    dominates the rows below it (each reflector then takes almost all of its
    column) and one whose columns span twelve orders of magnitude."""
    torch_cuda()
    g = np.random.default_rng(7)
    m, n = 1200, 300
    if case == "dominant_top":
        A = np.zeros((m, n))
        A[:n] = np.triu(g.standard_normal((n, n))) + 50.0 * np.eye(n)
        A[n:] = 1e-4 * g.standard_normal((m - n, n))
    elif case == "graded_columns":
        A = g.standard_normal((m, n)) * np.logspace(-6, 6, n)[None, :]
    else:
        A = g.standard_normal((m, n))
    A = np.asfortranarray(A)
    b = A @ g.standard_normal(n) + 1e-3 * g.standard_normal(m)
    X, it, berr, rc = tqr.tqr_solve_ls(to_dev(A), to_dev(b[:, None]), prec=tqr.TQR_PREC_FP32, tol=1e-12,
                                       maxit=0, nb=64, ib=16, check=False)
    assert it == 0
    eta = LS.backward_error(A, to_host(X)[:, 0], b)
    assert eta <= 50 * n * 2.0 ** -24, eta
    X2, it2, berr2, rc2 = tqr.tqr_solve_ls(to_dev(A), to_dev(b[:, None]), prec=tqr.TQR_PREC_FP32, tol=1e-12,
                                          maxit=40, nb=64, ib=16, check=False)
    assert rc2 == tqr.TQR_OK and LS.backward_error(A, to_host(X2)[:, 0], b) <= 1e-12

def test_solve_host_buffers():
    torch_cuda()
    A = inputs.normal_matrix(300, 100, 3)
    B = inputs.normal_matrix(300, 2, 4)
    X, it, berr, rc = tqr.tqr_solve_ls(A, B, nb=64, ib=16)
    assert rc == 0
    assert np.allclose(X, LS.lstsq(A, B), atol=1e-11)


def test_rank_deficient_reports_rank():
    torch_cuda()
    A = inputs.normal_matrix(200, 50, 5)
    A[:, 10] = A[:, 3]
    B = inputs.normal_matrix(200, 1, 6)
    X, it, berr, rc = tqr.tqr_solve_ls(to_dev(A), to_dev(B), nb=32, ib=8, check=False)
    assert rc == tqr.TQR_ERR_RANK


def test_full_size_least_squares_16384x4096():
    """The benchmark's least-squares launch (A 16384 x 4096 = U diag(sigma) V^T,
    kappa 1e2, nb 128, ib 16): the FP32-refined solution reaches backward
    error <= 1e-12, recomputed here in FP64 from the returned x, and agrees
    with the FP64 solve, which meets the same bound."""
    torch_cuda()
    A, b, _ = inputs.conditioned_ls_problem(16384, 4096, 1e2, seed=0)
    dA, db = to_dev(A), to_dev(b[:, None])
    X64, _, _, rc64 = tqr.tqr_solve_ls(dA, db, nb=128, ib=16, check=False)
    X32, it, berr, rc32 = tqr.tqr_solve_ls(dA, db, prec=tqr.TQR_PREC_FP32, tol=1e-12, maxit=30, nb=128, ib=16,
                                           check=False)
    assert rc64 == tqr.TQR_OK and rc32 == tqr.TQR_OK and it >= 1
    x64, x32 = to_host(X64)[:, 0], to_host(X32)[:, 0]
    assert LS.backward_error(A, x64, b) <= 1e-12
    assert LS.backward_error(A, x32, b) <= 1e-12
    assert np.linalg.norm(x32 - x64) <= 1e-12 * np.linalg.norm(x64)


def _fp64_bound(A, b, x):
    """First-order forward-error bound of a backward-stable FP64 LS solver:
    u kappa (2 + (kappa + 1) ||r|| / (||A|| ||x||))."""
    s = np.linalg.svd(A, compute_uv=False)
    kappa = s[0] / s[-1]
    r = b - A @ x
    return 2.0 ** -53 * kappa * (2.0 + (kappa + 1.0) * np.linalg.norm(r) / (s[0] * np.linalg.norm(x)))


def test_kappa_1e8_fp32_class_meets_the_fp64_contract():
    """kappa = 1e8 (the third class of the conditioned problems):
    kappa u_fp32 = 6, beyond the semi-normal and augmented refinements.  The
    FP32 class must still return status 0 with backward error <= 1e-12
    (recomputed here in FP64 by the oracle) and an x as accurate as an FP64
    solve -- reached by GMRES-IR or, where that stalls, by the FP64 re-solve
    (the info record says which)."""
    torch_cuda()
    A, b, _ = inputs.conditioned_ls_problem(2000, 500, 1e8, seed=1)
    X, it, berr, rc = tqr.tqr_solve_ls(to_dev(A), to_dev(b[:, None]), prec=tqr.TQR_PREC_FP32, tol=1e-12,
                                       maxit=30, nb=64, ib=16, check=False)
    info = tqr.tqr_ls_last_info()
    assert rc == tqr.TQR_OK, (rc, info)
    assert info["path"] in ("fp32_gmres", "fp64_fallback"), info
    x = to_host(X)[:, 0]
    assert LS.backward_error(A, x, b) <= 1e-12
    assert berr <= 1e-12
    xo = LS.lstsq(A, b)
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) <= 20.0 * _fp64_bound(A, b, xo), info


def test_gmres_ir_path_on_a_problem_it_can_finish():
    """kappa = 1e7 (kappa u_fp32 = 0.6): the augmented refinement cannot
    contract, GMRES-IR can; the result must come from GMRES-IR and meet the
    FP64 accuracy contract."""
    torch_cuda()
    A, b, _ = inputs.conditioned_ls_problem(1500, 300, 1e7, seed=3)
    X, it, berr, rc = tqr.tqr_solve_ls(to_dev(A), to_dev(b[:, None]), prec=tqr.TQR_PREC_FP32, tol=1e-12,
                                       maxit=30, nb=64, ib=16, check=False)
    info = tqr.tqr_ls_last_info()
    assert rc == tqr.TQR_OK, (rc, info)
    assert info["path"] == "fp32_gmres" and info["inner_iters"] >= 1, info
    x = to_host(X)[:, 0]
    assert LS.backward_error(A, x, b) <= 1e-12
    xo = LS.lstsq(A, b)
    assert np.linalg.norm(x - xo) / np.linalg.norm(xo) <= 20.0 * _fp64_bound(A, b, xo), info


@pytest.mark.parametrize("e", [531, -565])
def test_extreme_scaling(e):
    """A and b scaled by 2^531 (~1e160) and 2^-565 (~1e-170): the FP64 solve
    must return the unscaled problem's x (scaling both by a power of two
    leaves the LS solution unchanged) with a finite backward error, and the
    FP32 class -- whose ||A||_F is now outside FP32's range -- must be
    answered by the FP64 re-solve."""
    torch_cuda()
    A = inputs.normal_matrix(600, 150, 41)
    B = inputs.normal_matrix(600, 2, 42)
    X0, _, _, rc0 = tqr.tqr_solve_ls(to_dev(A), to_dev(B), nb=64, ib=16)
    s = 2.0 ** e
    X, it, berr, rc = tqr.tqr_solve_ls(to_dev(A * s), to_dev(B * s), nb=64, ib=16, check=False)
    assert rc == tqr.TQR_OK and np.isfinite(berr) and berr <= 1e-14
    x0, x = to_host(X0), to_host(X)
    assert np.max(np.abs(x - x0)) <= 1e-12 * np.abs(x0).max()
    X32, it, berr32, rc32 = tqr.tqr_solve_ls(to_dev(A * s), to_dev(B * s), prec=tqr.TQR_PREC_FP32, tol=1e-12,
                                             nb=64, ib=16, check=False)
    info = tqr.tqr_ls_last_info()
    assert rc32 == tqr.TQR_OK and info["path"] == "fp64_fallback", (rc32, info)
    assert info["fp32_status"] == tqr.TQR_ERR_UNSUPPORTED
    assert np.max(np.abs(to_host(X32) - x0)) <= 1e-12 * np.abs(x0).max()


@pytest.mark.parametrize("prec", [tqr.TQR_PREC_FP64, tqr.TQR_PREC_FP32])
def test_resident_handle_solves_repeated_right_hand_sides(prec):
    """tqr_ls_factor once, tqr_ls_solve for three right-hand-side blocks:
    each solution must match tqr_solve_ls on the same data (the same
    factorization arithmetic) and the oracle, and meet the backward error."""
    torch_cuda()
    A, _, _ = inputs.conditioned_ls_problem(1200, 300, 1e3, seed=5)
    dA = to_dev(A)
    h = tqr.LsHandle(dA, prec=prec, rhs_cap=4, nb=64, ib=16)
    dA.fill_(float("nan"))          # the handle keeps its own copy of A
    for k, nrhs in enumerate((1, 4, 2)):
        B = inputs.normal_matrix(1200, nrhs, 60 + k)
        X, info, rc = h.solve(to_dev(B), tol=1e-12)
        assert rc == tqr.TQR_OK, info
        Xs, _, _, rcs = tqr.tqr_solve_ls(to_dev(A), to_dev(B), prec=prec, tol=1e-12, nb=64, ib=16)
        x, xs, xo = to_host(X), to_host(Xs), LS.lstsq(A, B)
        assert np.max(np.abs(x - xs)) <= 1e-11 * np.abs(xs).max()
        assert np.max(np.abs(x - xo)) <= 1e-10 * np.abs(xo).max()
        assert LS.backward_error(A, x, B) <= 1e-12
        assert info["path"] == ("fp64" if prec == tqr.TQR_PREC_FP64 else "fp32_seminormal"), info
    h.release()
