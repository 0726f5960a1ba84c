"""GPU parity of the 2b x b bottom variant (tqr_factor_pairs /
tqr_apply_qt_pairs through the C ABI) against the oracle."""
import numpy as np
import pytest

from oracle import householder as H
from oracle import tiled as TL
from paper_0707_3548_gb300 import inputs, tqr
from tests.gpu_util import t_blocks, to_dev, to_host, torch_cuda

pytestmark = pytest.mark.gpu
U53 = 2.0 ** -53

SHAPES = [
    # m, n, nb, ib -- odd and even tile-row counts, ragged tails, ib = nb
    (512, 512, 128, 32),
    (700, 500, 128, 32),
    (1000, 300, 64, 16),
    (320, 256, 64, 64),
    (300, 600, 64, 16),
    (33, 17, 8, 4),
]


@pytest.mark.parametrize("m,n,nb,ib", SHAPES)
def test_pair_factor_matches_oracle(m, n, nb, ib):
    torch_cuda()
    A = inputs.normal_matrix(m, n, 201 + m + n)
    dA = to_dev(A)
    T = tqr.tqr_factor_pairs(dA, nb, ib)
    f = TL.tiled_qr_pairs(A, nb, ib)
    F = to_host(dA)
    assert np.max(np.abs(F - f.F)) <= 1e-11 * max(1.0, np.abs(f.F).max())
    Tg = t_blocks(T.cpu().numpy(), m, n, nb, ib)
    for key, Tk in f.T.items():
        assert np.max(np.abs(Tg[key] - Tk)) <= 1e-11 * max(1.0, np.abs(Tk).max()), key
    k = min(m, n)
    Ru = H.sign_normalize(H.r_factor(H.geqr2(A)[0]))[:k]
    assert np.linalg.norm(H.sign_normalize(np.triu(F))[:k] - Ru) / np.linalg.norm(Ru) <= 1e-11


@pytest.mark.parametrize("m,n,nb,ib,nrhs", [(700, 500, 128, 32, 3), (1000, 300, 64, 16, 40), (320, 256, 64, 64, 1)])
def test_pair_apply_matches_oracle(m, n, nb, ib, nrhs):
    A = inputs.normal_matrix(m, n, 211)
    B = inputs.normal_matrix(m, nrhs, 212)
    dA = to_dev(A)
    T = tqr.tqr_factor_pairs(dA, nb, ib)
    f = TL.tiled_qr_pairs(A, nb, ib)
    for trans, ref in (("T", TL.pairs_apply_qt(f, B)), ("N", TL.pairs_apply_q(f, B))):
        dB = to_dev(B)
        tqr.tqr_apply_qt_pairs(trans, dA, nb, ib, T, dB)
        assert np.max(np.abs(to_host(dB) - ref)) <= 1e-11 * max(1.0, np.abs(ref).max())


def test_pair_deterministic_across_schedules():
    A = inputs.normal_matrix(900, 700, 213)
    outs = []
    try:
        for policy, cap in ((-1, 0), (0, 0), (1, 0), (1, 3)):
            tqr.tqr_debug_set_schedule(policy, cap)
            dA = to_dev(A)
            T = tqr.tqr_factor_pairs(dA, 128, 32)
            outs.append((to_host(dA), T.cpu().numpy()))
    finally:
        tqr.tqr_debug_set_schedule(-1, 0)
    for F, T in outs[1:]:
        assert np.array_equal(F, outs[0][0]) and np.array_equal(T, outs[0][1])


def test_pair_host_path_equals_device_path():
    A = inputs.normal_matrix(400, 300, 214)
    dA = to_dev(A)
    T = tqr.tqr_factor_pairs(dA, 64, 16)
    hA = np.array(A, order="F", copy=True)
    hT = tqr.tqr_factor_pairs(hA, 64, 16)
    assert np.array_equal(hA, to_host(dA)) and np.array_equal(hT, T.cpu().numpy())


def test_full_size_sampled_pairs():
    """16384 x 16384 N(0,1), nb 128, ib 16 (the benchmark's launch): R's leading
    256 x 256 block equals the oracle's QR of A's first 256 columns, and Q R
    reproduces sampled columns of A."""
    torch = torch_cuda()
    m = n = 16384
    A = inputs.normal_matrix(m, n, 0)
    dA = to_dev(A)
    T = tqr.tqr_factor_pairs(dA, 128, 16)
    torch.cuda.synchronize()
    lead = dA[:256, :256].cpu().numpy()
    Fo, _ = H.geqr2(A[:, :256])
    assert np.linalg.norm(H.sign_normalize(np.triu(lead)) - H.sign_normalize(np.triu(Fo[:256]))) / \
        np.linalg.norm(Fo[:256]) <= 1e-11
    cols = [0, 1, 127, 128, 8191, 16383]
    Rs = tqr.colmajor(torch.triu(dA)[:, cols].contiguous())
    tqr.tqr_apply_qt_pairs("N", dA, 128, 16, T, Rs)
    err = np.linalg.norm(to_host(Rs) - A[:, cols]) / np.linalg.norm(A[:, cols])
    assert err <= 10 * n * U53


def test_full_size_every_column_and_sampled_gram_entries():
    """16384 x 16384, nb 128, ib 16 (the benchmark's launch), checked in
    every block of R with identities that hold at any size: Q is orthogonal,
    so ||R e_j|| = ||A e_j|| for every column j, and (R^T R)(i, j) =
    (A^T A)(i, j) for every pair -- here 400 pairs drawn over the whole
    matrix, interior and trailing blocks included -- within a few units of
    FP64 rounding relative to the column norms (1e4 u; a wrong block would
    be off by O(1))."""
    torch = torch_cuda()
    m = n = 16384
    A = inputs.normal_matrix(m, n, 0)
    dA = to_dev(A)
    tqr.tqr_factor_pairs(dA, 128, 16)
    torch.cuda.synchronize()
    R = torch.triu(dA)
    rn = torch.linalg.vector_norm(R, dim=0).cpu().numpy()
    an = np.linalg.norm(A, axis=0)
    assert np.max(np.abs(rn - an) / an) <= 1e4 * U53
    g = inputs.rng(5)
    ii = g.integers(0, n, 400)
    jj = g.integers(0, n, 400)
    Rc = R.cpu().numpy()
    for i, j in zip(ii, jj):
        rr = Rc[:, i] @ Rc[:, j]
        aa = A[:, i] @ A[:, j]
        assert abs(rr - aa) <= 1e4 * U53 * an[i] * an[j], (i, j, rr, aa)
    # the stored factor: reflectors below the diagonal, R on and above; the
    # returned R (upper part) has its own diagonal entries nonzero
    assert np.all(np.abs(np.diag(Rc)) > 0)


def test_pair_and_flat_plans_do_not_mix():
    """Both variants of one shape, alternately: each must run its own task
    list (the plan cache keys on the variant)."""
    A = inputs.normal_matrix(512, 512, 215)
    f_flat = TL.tiled_qr(A, 128, 32)
    f_pair = TL.tiled_qr_pairs(A, 128, 32)
    for _ in range(2):
        dA = to_dev(A)
        tqr.tqr_factor_pairs(dA, 128, 32)
        assert np.max(np.abs(to_host(dA) - f_pair.F)) <= 1e-11 * np.abs(f_pair.F).max()
        dA = to_dev(A)
        tqr.tqr_factor(dA, 128, 32)
        assert np.max(np.abs(to_host(dA) - f_flat.F)) <= 1e-11 * np.abs(f_flat.F).max()


@pytest.mark.parametrize("m,n,nb,ib", [(1, 1, 8, 8), (5, 3, 8, 4), (8, 8, 8, 2), (17, 40, 8, 4), (24, 1, 8, 8),
                                       (40, 17, 8, 8), (100, 7, 16, 4)])
def test_pair_tiny_and_degenerate_shapes(m, n, nb, ib):
    torch_cuda()
    A = inputs.uniform_matrix(m, n, 221 + m + n)
    dA = to_dev(A)
    T = tqr.tqr_factor_pairs(dA, nb, ib)
    f = TL.tiled_qr_pairs(A, nb, ib)
    assert np.max(np.abs(to_host(dA) - f.F)) <= 1e-12 * max(1.0, np.abs(f.F).max())
    B = inputs.uniform_matrix(m, 2, 222)
    dB = to_dev(B)
    tqr.tqr_apply_qt_pairs("T", dA, nb, ib, T, dB)
    assert np.max(np.abs(to_host(dB) - TL.pairs_apply_qt(f, B))) <= 1e-12 * max(1.0, np.abs(B).max())
