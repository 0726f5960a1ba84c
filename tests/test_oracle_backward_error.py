"""Pins for the oracle's least-squares backward error.

The paper defines no backward error; the reading used throughout is the
normwise ratio
    eta(x) = ||A^T r||_2 / (||A||_F (||A||_F ||x||_2 + ||b||_2)),  r = b - A x,
taken as the maximum over right-hand sides.  The pins below fix it by values
worked out by hand from that definition (not by re-running the formula),
by invariances that any correct implementation keeps, and by planted
mistakes that must fail them: the spectral norm in place of the Frobenius
norm, a dropped ||b|| or ||x|| term, ||A||_F squared in the outer factor,
||r|| in place of ||A^T r||, and a sum over right-hand sides in place of the
maximum."""
import math

import numpy as np
import pytest

from oracle import lstsq as L
from paper_0707_3548_gb300 import inputs

# ---- hand-worked cases ---------------------------------------------------------
# (1) A = [1; 0], b = [1; 1], x = 0:  r = [1; 1], A^T r = 1, ||A||_F = 1,
#     ||x|| = 0, ||b|| = sqrt(2):  eta = 1 / (1 * (0 + sqrt(2))) = 1/sqrt(2).
# (2) A = [[3, 0], [0, 4], [0, 0]] (||A||_F = 5, ||A||_2 = 4), x = [0; 1],
#     b = [2; 4; 4] (||b|| = 6):  A x = [0; 4; 0], r = [2; 0; 4],
#     A^T r = [6; 0]:  eta = 6 / (5 * (5 * 1 + 6)) = 6/55.
# (3) the same A with two right-hand sides: column 1 as in (2), column 2
#     x = [0; 0], b = [1; 0; 0]:  r = b, A^T r = [3; 0],
#     eta_2 = 3 / (5 * (0 + 1)) = 3/5;  the result is max(6/55, 3/5) = 3/5.
A2 = np.array([[3.0, 0.0], [0.0, 4.0], [0.0, 0.0]])
CASES = [
    (np.array([[1.0], [0.0]]), np.array([0.0]), np.array([1.0, 1.0]), 1.0 / math.sqrt(2.0)),
    (A2, np.array([0.0, 1.0]), np.array([2.0, 4.0, 4.0]), 6.0 / 55.0),
    (A2, np.array([[0.0, 0.0], [1.0, 0.0]]), np.array([[2.0, 1.0], [4.0, 0.0], [4.0, 0.0]]), 3.0 / 5.0),
]


def _pins_hold(fn):
    """True when fn meets every pin: the hand-worked values, the scaling and
    orthogonal invariances, and zero exactly at a solution of the normal
    equations whatever the size of the residual."""
    try:
        for A, x, b, eta in CASES:
            if not abs(fn(A, x, b) - eta) <= 1e-15 * eta:
                return False
        A, b, _ = inputs.conditioned_ls_problem(40, 8, 1e3, seed=11)
        x = np.linalg.lstsq(A, b, rcond=None)[0] + 1e-6 * inputs.normal_matrix(8, 1, 12)[:, 0]
        e0 = fn(A, x, b)
        if not e0 > 0:
            return False
        # eta(alpha A, x, alpha b) = eta(A, x, b): r and A^T r scale by alpha and
        # alpha^2, the denominator by alpha^2 (powers of two scale exactly)
        if not abs(fn(8.0 * A, x, 8.0 * b) - e0) <= 1e-12 * e0:
            return False
        # eta(A, beta x, beta b) = eta(A, x, b): numerator and denominator scale by beta
        if not abs(fn(A, 0.125 * x, 0.125 * b) - e0) <= 1e-12 * e0:
            return False
        # an orthogonal change of rows (a permutation with signs) changes nothing
        # but the order of the sums (A^T r cancels to ~1e-7 of its terms here)
        P = np.eye(40)[::-1] * np.where(np.arange(40) % 3 == 0, -1.0, 1.0)[:, None]
        if not abs(fn(P @ A, x, P @ b) - e0) <= 1e-9 * e0:
            return False
        # b = A y + z with A^T z = 0 exactly (z built orthogonal to A's columns
        # in exact integer arithmetic): x = y gives A^T r = 0 however large r is
        Ai = np.array([[1.0, 0.0], [1.0, 1.0], [0.0, 1.0], [1.0, 2.0]])
        z = np.array([1.0, -2.0, 0.0, 1.0])     # A^T z = [1 - 2 + 1, -2 + 2] = 0
        assert np.all(Ai.T @ z == 0.0)
        y = np.array([2.0, -3.0])
        if fn(Ai, y, Ai @ y + 5.0 * z) != 0.0:
            return False
    except (ValueError, ZeroDivisionError, FloatingPointError):
        return False
    return True


def test_oracle_backward_error_meets_the_pins():
    assert _pins_hold(L.backward_error)


@pytest.mark.parametrize("A,x,b,eta", CASES)
def test_hand_worked_values(A, x, b, eta):
    assert L.backward_error(A, x, b) == pytest.approx(eta, rel=1e-15)


# ---- planted mistakes ----------------------------------------------------------
def _eta_variant(norm_a, numerator, outer_square=False, drop_b=False, drop_x=False, combine=max):
    def fn(A, x, b):
        A = np.asarray(A, dtype=np.float64)
        x = np.asarray(x, dtype=np.float64)
        b = np.asarray(b, dtype=np.float64)
        if x.ndim == 1:
            x, b = x[:, None], b[:, None]
        nA = norm_a(A)
        vals = []
        for c in range(x.shape[1]):
            r = b[:, c] - A @ x[:, c]
            num = numerator(A, r)
            inner = (0.0 if drop_x else nA * np.linalg.norm(x[:, c])) + (0.0 if drop_b else np.linalg.norm(b[:, c]))
            vals.append(num / ((nA * nA if outer_square else nA) * inner))
        return combine(vals)
    return fn


def _fro(A):
    return np.linalg.norm(A, "fro")


def _atr(A, r):
    return np.linalg.norm(A.T @ r)


def test_correct_variant_meets_the_pins():
    # the variant builder itself, unmutated, is the definition
    assert _pins_hold(_eta_variant(_fro, _atr))


@pytest.mark.parametrize("name,fn", [
    ("spectral norm for ||A||", _eta_variant(lambda A: np.linalg.norm(A, 2), _atr)),
    ("||b|| term dropped", _eta_variant(_fro, _atr, drop_b=True)),
    ("||A|| ||x|| term dropped", _eta_variant(_fro, _atr, drop_x=True)),
    ("||A||_F squared outside", _eta_variant(_fro, _atr, outer_square=True)),
    ("||r|| for ||A^T r||", _eta_variant(_fro, lambda A, r: np.linalg.norm(r))),
    ("sum over right-hand sides", _eta_variant(_fro, _atr, combine=sum)),
    ("root of summed squared column norms squared", _eta_variant(
        lambda A: math.sqrt(sum(np.linalg.norm(A[:, c]) ** 4 for c in range(A.shape[1]))), _atr)),
])
def test_planted_mistake_fails_the_pins(name, fn):
    with np.errstate(divide="ignore", invalid="ignore"):
        assert not _pins_hold(fn), name
