"""Pins for the oracle's 2b x b bottom variant (Section 3.2's remark on
non-square blocks): the factors against the unblocked Householder oracle and
identities of Q, the degenerate cases that are exactly Algorithm 1, and the
operation count against the 12.5 % the paper prints."""
import numpy as np
import pytest

from oracle import dag as D
from oracle import householder as H
from oracle import tiled as TL
from paper_0707_3548_gb300 import inputs

U53 = 2.0 ** -53


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_tall_kernel_counts_reduce_to_section_3_2():
    assert D.tall_kernel_flops_b3(D.TSQRT, 1) == pytest.approx(10.0 / 3.0)
    assert D.tall_kernel_flops_b3(D.SSRFB, 1) == pytest.approx(5.0)
    assert D.opcount_pairs(2, 2) == pytest.approx(D.opcount_tiles(2, 2))   # one bottom row: no pair


def test_pair_opcount_is_twelve_and_a_half_percent_above_lapack():
    # Section 3.2 / Section 5: 2b x b blocks reduce the 25 % overhead to 12.5 %
    for p, q in ((400, 400), (800, 200)):
        b = 1.0
        ratio = D.opcount_pairs(p, q) * b ** 3 / D.lapack_flops(p * b, q * b)
        assert ratio == pytest.approx(1.125, rel=0.02)
        assert D.opcount_tiles(p, q) / D.lapack_flops(p, q) == pytest.approx(1.25, rel=0.02)


def test_group_cover_rows_once():
    for p in range(1, 12):
        for k in range(p):
            rows = [r for _, g in TL.pair_groups(k, p) for r in g]
            assert rows == list(range(k + 1, p))
            assert all(len(g) == 2 for _, g in TL.pair_groups(k, p)[:-1])


@pytest.mark.parametrize("m,n,nb,ib", [(96, 48, 16, 4), (100, 60, 16, 8), (64, 64, 16, 16), (150, 40, 16, 4),
                                       (33, 17, 8, 2), (70, 90, 16, 8)])
def test_pair_factors_match_unblocked_qr(m, n, nb, ib):
    A = inputs.normal_matrix(m, n, m + 3 * n)
    f = TL.tiled_qr_pairs(A, nb, ib)
    k = min(m, n)
    Ru = H.sign_normalize(H.r_factor(H.geqr2(A)[0]))[:k]
    assert _rel(H.sign_normalize(f.R)[:k], Ru) <= 50 * n * U53
    assert np.all(np.tril(f.R, -1) == 0)
    R = np.zeros((m, n))
    R[:k] = f.R[:k]
    assert _rel(TL.pairs_apply_q(f, R), A) <= 10 * n * U53
    Q = TL.pairs_apply_q(f, np.eye(m))
    assert np.linalg.norm(Q.T @ Q - np.eye(m)) <= 10 * m * U53
    B = inputs.normal_matrix(m, 3, 5)
    assert _rel(TL.pairs_apply_qt(f, TL.pairs_apply_q(f, B)), B) <= 10 * m * U53


def test_two_tile_rows_are_exactly_algorithm_1():
    A = inputs.normal_matrix(32, 40, 6)
    f = TL.tiled_qr_pairs(A, 16, 4)
    g = TL.tiled_qr(A, 16, 4)
    assert np.array_equal(f.Ap, g.Ap)


def test_misplaced_pair_reflectors_are_caught():
    """Planted mistake: the two halves of a pair's reflectors stored in each
    other's tiles must fail Q R = A."""
    m, n, nb, ib = 80, 32, 16, 4
    A = inputs.normal_matrix(m, n, 7)
    f = TL.tiled_qr_pairs(A, nb, ib)
    bad = TL.PairFactors(m, n, nb, ib, f.Ap.copy(), dict(f.T))
    t1, t2 = bad.tile(1, 0).copy(), bad.tile(2, 0).copy()
    bad.tile(1, 0)[:], bad.tile(2, 0)[:] = t2, t1
    R = np.zeros((m, n))
    R[:n] = f.R[:n]
    assert _rel(TL.pairs_apply_q(bad, R), A) > 1e-3
