"""Planted mistakes in the oracle (on the CPU) must be caught by the pins.

Each case swaps one oracle function for a plausibly wrong variant (a
transposed operand, a dropped term, a wrong sign or index) and checks that
the invariant pins reject the result."""
import numpy as np
import pytest

from oracle import householder as H
from oracle import tiled as TL
from paper_0707_3548_gb300 import inputs

U53 = 2.0 ** -53


def _pins_hold(m=40, n=33, nb=8, ib=4):
    A = inputs.normal_matrix(m, n, 123)
    f = TL.tiled_qr(A, nb, ib)
    Q = TL.form_q(f)
    R = f.R
    tol = 10 * max(m, n) * U53
    ok_qr = np.linalg.norm(Q @ R - A) / np.linalg.norm(A) <= tol
    ok_orth = np.linalg.norm(np.eye(m) - Q.T @ Q) <= tol
    Fu, _ = H.geqr2(A)
    ok_unb = np.linalg.norm(H.sign_normalize(R)[:n] - H.sign_normalize(H.r_factor(Fu))[:n]) <= 1e-12 * np.linalg.norm(A)
    return ok_qr and ok_orth and ok_unb


def test_unmutated_oracle_passes():
    assert _pins_hold()


def _larfb_impl(C, Fkk, Tkk, ib, trans, transpose_T):
    C = np.array(C, dtype=np.float64, copy=True)
    nb = Fkk.shape[0]
    blocks = list(range(0, nb, ib))
    if not trans:
        blocks.reverse()
    for l0 in blocks:
        V = H.unit_lower(Fkk[l0:, l0:l0 + ib], ib)
        Tl = Tkk[:, l0:l0 + ib]
        op = Tl.T if (trans == transpose_T) else Tl
        C[l0:, :] -= V @ (op @ (V.T @ C[l0:, :]))
    return C


def test_mutation_transposed_T_in_larfb(monkeypatch):
    monkeypatch.setattr(TL, "larfb", lambda C, F, T, ib, trans=True: _larfb_impl(C, F, T, ib, trans, transpose_T=False))
    assert not _pins_hold()


def test_mutation_dropped_identity_term_in_ssrfb(monkeypatch):
    def bad(Akj, Aij, Vik, Tik, ib, trans=True):
        nb = Vik.shape[0]
        C = np.vstack([Akj, Aij]).astype(np.float64)
        blocks = list(range(0, nb, ib))
        if not trans:
            blocks.reverse()
        for l0 in blocks:
            Vfull = TL._stacked_v(Vik[:, l0:l0 + ib], l0, ib, nb)
            Vfull[:nb] = 0.0                      # drops the [I] part of [I; V]
            Tl = Tik[:, l0:l0 + ib]
            op = Tl.T if trans else Tl
            C -= Vfull @ (op @ (Vfull.T @ C))
        return C[:nb].copy(), C[nb:].copy()
    monkeypatch.setattr(TL, "ssrfb", bad)
    assert not _pins_hold()


def test_mutation_larft_wrong_sign(monkeypatch):
    def bad(V, tau):
        k = len(tau)
        T = np.zeros((k, k))
        for i in range(k):
            T[i, i] = tau[i]
            if i > 0:
                T[:i, i] = +tau[i] * (T[:i, :i] @ (V[:, :i].T @ V[:, i]))
        return T
    monkeypatch.setattr(TL, "larft", bad)
    assert not _pins_hold()


def test_mutation_tsqrt_off_by_one_column(monkeypatch):
    def bad(Rkk, Aik, ib):
        R = np.array(Rkk, dtype=np.float64, copy=True)
        A = np.array(Aik, dtype=np.float64, copy=True)
        nb = R.shape[0]
        T = np.zeros((ib, nb))
        for l0 in range(0, nb, ib):
            l1 = l0 + ib
            tau = np.zeros(ib)
            for c in range(l0, l1):
                t, v2, beta = H.householder(R[c, c], A[:, c])
                R[c, c] = beta
                A[:, c] = v2
                tau[c - l0] = t
                if t != 0.0 and c + 2 < l1:           # skips column c+1
                    w = R[c, c + 2:l1] + v2 @ A[:, c + 2:l1]
                    R[c, c + 2:l1] -= t * w
                    A[:, c + 2:l1] -= t * np.outer(v2, w)
            Vfull = TL._stacked_v(A[:, l0:l1], l0, ib, nb)
            Tl = H.larft(Vfull, tau)
            T[:, l0:l1] = Tl
            if l1 < nb:
                C = np.vstack([R[:, l1:], A[:, l1:]])
                C -= Vfull @ (Tl.T @ (Vfull.T @ C))
                R[l0:l1, l1:] = C[l0:l1, :]
                A[:, l1:] = C[nb:, :]
        return R, A, T
    monkeypatch.setattr(TL, "tsqrt", bad)
    assert not _pins_hold()


def test_mutation_reflector_missing_scaling(monkeypatch):
    orig = H.householder

    def bad(alpha, x2):
        tau, v2, beta = orig(alpha, x2)
        return tau, v2 * 1.0000001, beta
    monkeypatch.setattr(TL, "householder", bad)
    assert not _pins_hold()


# ---- least-squares refinement ------------------------------------------------
from oracle import lstsq as LSQ  # noqa: E402


def _seminormal_pins_hold():
    """The semi-normal pins: with the exact R one correction reaches the LS
    solution, and with an R perturbed by 1e-7 the backward error falls
    geometrically to the rounding level."""
    A, b, _ = inputs.conditioned_ls_problem(120, 20, 1e2, seed=3)
    x_ref = np.linalg.lstsq(A, b, rcond=None)[0]
    R = np.linalg.qr(A, mode="r")
    try:
        x, it, hist = LSQ.seminormal_refinement(A, b, R, tol=1e-15, maxit=3)
        ok_exact = hist[-1] <= 1e-15 and np.linalg.norm(x - x_ref) <= 1e-10 * np.linalg.norm(x_ref)
        E = 1e-7 * np.linalg.norm(A, 2) * inputs.normal_matrix(120, 20, 4) / np.sqrt(120)
        Rp = np.linalg.qr(A + E, mode="r")
        x, it, hist = LSQ.seminormal_refinement(A, b, Rp, tol=1e-14, maxit=20)
        ok_pert = hist[-1] <= 1e-14 and it <= 6
    except (ValueError, np.linalg.LinAlgError, FloatingPointError):
        return False
    return bool(ok_exact and ok_pert)


def test_unmutated_seminormal_refinement_passes():
    assert _seminormal_pins_hold()


def test_mutation_seminormal_without_the_transposed_solve(monkeypatch):
    # R^-1 R^-1 A^T e in place of R^-1 R^-T A^T e
    monkeypatch.setattr(LSQ, "forward_substitution_rt", LSQ.back_substitution)
    assert not _seminormal_pins_hold()


def test_mutation_seminormal_with_the_residual_sign_flipped(monkeypatch):
    orig = LSQ.back_substitution

    def flipped(R, C):
        return -orig(R, C)

    monkeypatch.setattr(LSQ, "back_substitution", flipped)
    assert not _seminormal_pins_hold()


def _augmented_pins_hold(solver_cls=LSQ.QRSolver):
    """The augmented-system pins: with an R and Q perturbed by 1e-7 the
    refinement reaches backward error 1e-14 and the LS solution."""
    A, b, _ = inputs.conditioned_ls_problem(150, 25, 1e2, seed=5)
    x_ref = np.linalg.lstsq(A, b, rcond=None)[0]
    E = 1e-7 * np.linalg.norm(A, 2) * inputs.normal_matrix(150, 25, 6) / np.sqrt(150)
    try:
        x, r, it, hist = LSQ.augmented_refinement(A, b, solver_cls(A + E), tol=1e-14, maxit=20)
    except (ValueError, np.linalg.LinAlgError, FloatingPointError):
        return False
    return bool(hist[-1] <= 1e-14 and np.linalg.norm(x - x_ref) <= 1e-10 * np.linalg.norm(x_ref))


def test_unmutated_augmented_refinement_passes():
    assert _augmented_pins_hold()


def test_mutation_augmented_with_h_added(monkeypatch):
    # dx = R^-1 (d1 + h) in place of R^-1 (d1 - h)
    orig = LSQ.forward_substitution_rt
    monkeypatch.setattr(LSQ, "forward_substitution_rt", lambda R, G: -orig(R, G))
    assert not _augmented_pins_hold()


def test_mutation_augmented_with_q_and_qt_swapped():
    class Swapped(LSQ.QRSolver):
        def qt(self, B):
            return super().q(B)

        def q(self, B):
            return super().qt(B)

    assert not _augmented_pins_hold(Swapped)
