"""GPU parity of the reduction-tree variant against the oracle."""
import numpy as np
import pytest

from oracle import householder as H
from oracle import lstsq as LS
from oracle import tiled as TL
from paper_0707_3548_gb300 import inputs, tqr
from tests.gpu_util import t_blocks, to_dev, to_host, torch_cuda

pytestmark = pytest.mark.gpu


def _tree(A, nb, ib, D):
    torch_cuda()
    dA = to_dev(A)
    T, d = tqr.tqr_factor_tree(dA, nb, ib, D)
    return to_host(dA), T.cpu().numpy(), d, dA, T


@pytest.mark.parametrize("m,n,nb,ib,D", [(1000, 200, 64, 16, 1), (1000, 200, 64, 32, 2), (900, 150, 32, 8, 3),
                                          (600, 600, 64, 16, 2), (700, 130, 128, 32, 1), (333, 50, 16, 8, 4)])
def test_tree_factor_matches_oracle(m, n, nb, ib, D):
    A = inputs.normal_matrix(m, n, m + n + D)
    F, Tflat, d, _, _ = _tree(A, nb, ib, D)
    assert d == D
    f = TL.tree_qr(A, nb, ib, D)
    assert np.max(np.abs(F - f.F)) <= 1e-11 * np.abs(f.F).max()
    half = Tflat.size // 2
    T1 = t_blocks(Tflat[:half], m, n, nb, ib)
    T2 = t_blocks(Tflat[half:], m, n, nb, ib)
    for key, T in f.T.items():
        assert np.max(np.abs(T1[key] - T)) <= 1e-11 * max(1.0, np.abs(T).max()), key
    for key, T in f.T2.items():
        assert np.max(np.abs(T2[key] - T)) <= 1e-11 * max(1.0, np.abs(T).max()), key
    k = min(m, n)
    Ru = H.sign_normalize(H.r_factor(H.geqr2(A)[0]))[:k]
    assert np.linalg.norm(H.sign_normalize(np.triu(F))[:k] - Ru) / np.linalg.norm(Ru) <= 1e-11


@pytest.mark.parametrize("D", [1, 3])
def test_tree_apply_matches_oracle(D):
    m, n, nb, ib, nrhs = 800, 120, 32, 8, 5
    A = inputs.normal_matrix(m, n, 4)
    B = inputs.normal_matrix(m, nrhs, 5)
    _, _, _, dA, T = _tree(A, nb, ib, D)
    f = TL.tree_qr(A, nb, ib, D)
    for trans, ref in (("T", TL.tree_apply_qt(f, B)), ("N", TL.tree_apply_q(f, B))):
        dB = to_dev(B)
        tqr.tqr_apply_qt_tree(trans, dA, nb, ib, D, T, dB)
        assert np.max(np.abs(to_host(dB) - ref)) <= 1e-11 * np.abs(ref).max()


def test_tree_auto_domain_tall_skinny_and_determinism():
    m, n, nb, ib = 8192, 256, 64, 16
    A = inputs.normal_matrix(m, n, 6)
    F1, T1, d, _, _ = _tree(A, nb, ib, 0)
    assert 1 <= d < m // nb            # a tree is chosen for 128 x 4 tiles
    try:
        tqr.tqr_debug_set_schedule(0, 7)
        F2, T2, _, _, _ = _tree(A, nb, ib, d)
    finally:
        tqr.tqr_debug_set_schedule(-1, 0)
    assert np.array_equal(F1, F2) and np.array_equal(T1, T2)
    Fo, _ = H.geqr2(A[:, :64])
    Rl = H.sign_normalize(np.triu(F1[:64, :64]))
    assert np.linalg.norm(Rl - H.sign_normalize(np.triu(Fo[:64]))) / np.linalg.norm(Fo[:64]) <= 1e-11


@pytest.mark.parametrize("prec", [tqr.TQR_PREC_FP64, tqr.TQR_PREC_FP32])
def test_tall_least_squares_through_tree(prec):
    torch_cuda()
    A = inputs.normal_matrix(6000, 120, 7)
    b = inputs.normal_matrix(6000, 2, 8)
    X, it, berr, rc = tqr.tqr_solve_ls(to_dev(A), to_dev(b), prec=prec, nb=32, ib=16)
    assert rc == 0 and berr <= 1e-12
    assert np.allclose(to_host(X), LS.lstsq(A, b), atol=1e-11)


def test_full_size_sampled_tall_skinny_tree():
    """65536 x 2048 N(0,1), nb 128, ib 16, the library's domain choice (the
    benchmark's tall-skinny launch): R's leading 256 x 256 block equals the
    oracle's QR of A's first 256 columns up to row signs, and Q R reproduces
    sampled columns of A."""
    torch = torch_cuda()
    m, n = 65536, 2048
    A = inputs.normal_matrix(m, n, 0)
    dA = to_dev(A)
    T, D = tqr.tqr_factor_tree(dA, 128, 16, 0)
    torch.cuda.synchronize()
    assert D > 0
    lead = dA[:256, :256].cpu().numpy()
    Fo, _ = H.geqr2(A[:, :256])
    assert np.linalg.norm(H.sign_normalize(np.triu(lead)) - H.sign_normalize(np.triu(Fo[:256]))) / \
        np.linalg.norm(Fo[:256]) <= 1e-11
    cols = [0, 1, 127, 128, 1023, 2047]
    Rs = torch.zeros((m, len(cols)), dtype=torch.float64, device="cuda")
    Rs[:n] = torch.triu(dA[:n, :n])[:, cols]
    Rs = tqr.colmajor(Rs)
    tqr.tqr_apply_qt_tree("N", dA, 128, 16, D, T, Rs)
    err = np.linalg.norm(to_host(Rs) - A[:, cols]) / np.linalg.norm(A[:, cols])
    assert err <= 10 * m * 2.0 ** -53
