"""The multithreaded C tiled QR (oracle/ctiled.c, the CPU baseline) against
the NumPy oracle, which its own pins fix.

- F (R and the tiled V) and every T block equal the NumPy oracle's
  Algorithm 1 within rounding, for square, tall, wide and ragged shapes and
  several (nb, ib), including ib = nb (the paper's unblocked kernels).
- Each tile's sequence of updates is fixed by the DAG, so the result does
  not depend on the schedule: 1, 3 and 8 threads give the same bits.
- R equals LAPACK's R after the sign fix (a third opinion)."""
import numpy as np
import pytest

from oracle import ctiled as C
from oracle import householder as H
from oracle import tiled as TL
from paper_0707_3548_gb300 import inputs


def _t_flat(f, m, n, nb, ib):
    p, q = TL.grid(m, n, nb)
    out = []
    for k in range(min(p, q)):
        for i in range(k, p):
            out.append(np.asarray(f.T[(i, k)]).T.ravel())   # ib x nb, column-major
    return np.concatenate(out)


@pytest.mark.parametrize("m,n,nb,ib", [(64, 64, 16, 4), (100, 37, 16, 8), (37, 100, 16, 16), (130, 130, 32, 8),
                                       (200, 90, 24, 6), (48, 48, 48, 48), (257, 129, 32, 32)])
def test_matches_numpy_oracle(m, n, nb, ib):
    A = inputs.normal_matrix(m, n, 71)
    F, T, _ = C.tiled_qr(A, nb, ib, threads=4)
    f = TL.tiled_qr(A, nb, ib)
    scale = np.abs(f.F).max()
    assert np.max(np.abs(F - f.F)) <= 1e-13 * scale
    Tr = _t_flat(f, m, n, nb, ib)
    assert T.shape == Tr.shape
    assert np.max(np.abs(T - Tr)) <= 1e-13 * max(1.0, np.abs(Tr).max())


def test_schedule_does_not_change_a_bit():
    A = inputs.normal_matrix(300, 220, 72)
    F1, T1, _ = C.tiled_qr(A, 32, 8, threads=1)
    for th in (3, 8):
        F, T, _ = C.tiled_qr(A, 32, 8, threads=th)
        assert np.array_equal(F, F1) and np.array_equal(T, T1)


def test_r_matches_lapack_after_sign_fix():
    A = inputs.normal_matrix(400, 300, 73)
    F, _, _ = C.tiled_qr(A, 64, 16, threads=4)
    R = H.sign_normalize(np.triu(F)[:300])
    Rl = H.sign_normalize(np.linalg.qr(A, mode="r"))
    assert np.linalg.norm(R - Rl) <= 1e-13 * np.linalg.norm(Rl)


def test_rejects_invalid_arguments():
    with pytest.raises(ValueError):
        C.tiled_qr(np.zeros((8, 8)), 8, 3)      # ib does not divide nb
