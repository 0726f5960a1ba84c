"""GPU parity of op(Q) C, C op(Q) and the explicit Q columns (tqr_ormqr /
tqr_orgqr through the C ABI) against the oracle."""
import numpy as np
import pytest

from oracle import tiled as TL
from paper_0707_3548_gb300 import inputs, tqr
from tests.gpu_util import to_dev, to_host, torch_cuda

pytestmark = pytest.mark.gpu
U53 = 2.0 ** -53


def _maxrel(got, ref):
    return np.max(np.abs(got - ref)) / max(1.0, np.abs(ref).max()) if ref.size else 0.0


def _factor(A, nb, ib, D=0):
    torch_cuda()
    dA = to_dev(A)
    if D:
        T, D = tqr.tqr_factor_tree(dA, nb, ib, D)
        f = TL.tree_qr(A, nb, ib, D)
    else:
        T = tqr.tqr_factor(dA, nb, ib)
        f = TL.tiled_qr(A, nb, ib)
    return dA, T, D, f


ORG = [
    # m, n, nb, ib, ncols -- several tiles, ragged tails, m < n, partial Q
    (700, 500, 128, 32, 500),
    (300, 300, 64, 16, 300),
    (257, 129, 64, 64, 257),
    (1000, 77, 128, 16, 77),
    (33, 17, 8, 4, 20),
    (130, 200, 64, 16, 130),
    (640, 640, 64, 16, 1),
]


@pytest.mark.parametrize("m,n,nb,ib,ncols", ORG)
def test_orgqr_matches_oracle(m, n, nb, ib, ncols):
    A = inputs.normal_matrix(m, n, 31 + m + n)
    dA, T, D, f = _factor(A, nb, ib)
    Q = to_host(tqr.tqr_orgqr(dA, nb, ib, T, ncols))
    ref = TL.orgqr(f, ncols)
    assert _maxrel(Q, ref) <= 1e-11
    assert np.linalg.norm(Q.T @ Q - np.eye(ncols)) <= 10 * m * U53


@pytest.mark.parametrize("m,n,nb,ib,D", [(1024, 96, 32, 8, 2), (700, 130, 64, 16, 3), (512, 512, 64, 16, 1)])
def test_orgqr_tree_matches_oracle(m, n, nb, ib, D):
    A = inputs.normal_matrix(m, n, 41)
    dA, T, D, f = _factor(A, nb, ib, D)
    for ncols in (n, m):
        Q = to_host(tqr.tqr_orgqr(dA, nb, ib, T, ncols, D=D))
        assert _maxrel(Q, TL.orgqr(f, ncols)) <= 1e-11


@pytest.mark.parametrize("m,n,nb,ib,D", [(700, 500, 128, 32, 0), (300, 600, 64, 16, 0), (257, 129, 64, 64, 0),
                                         (1024, 96, 32, 8, 2)])
@pytest.mark.parametrize("side,trans", [("L", "N"), ("L", "T"), ("R", "N"), ("R", "T")])
def test_ormqr_matches_oracle(m, n, nb, ib, D, side, trans):
    A = inputs.normal_matrix(m, n, 51)
    dA, T, D, f = _factor(A, nb, ib, D)
    C = inputs.normal_matrix(m, 37, 52) if side == "L" else inputs.normal_matrix(45, m, 53)
    dC = to_dev(C)
    tqr.tqr_ormqr(side, trans, dA, nb, ib, T, dC, D=D)
    assert _maxrel(to_host(dC), TL.ormqr(f, side, trans, C)) <= 1e-11


def test_ormqr_right_with_leading_dimension_and_host_path():
    """C as a block of a larger column-major array (ldc > mc), and host
    operands staged by the library: both equal the device result."""
    torch = torch_cuda()
    m, n, nb, ib = 300, 200, 64, 16
    A = inputs.normal_matrix(m, n, 61)
    dA, T, _, f = _factor(A, nb, ib)
    C = inputs.normal_matrix(70, m, 62)
    big = tqr.colmajor(torch.zeros((100, m), dtype=torch.float64, device="cuda"))
    big[10:80] = torch.from_numpy(C).cuda()
    sub = big[10:80]
    tqr.tqr_ormqr("R", "T", dA, nb, ib, T, sub)
    ref = TL.ormqr(f, "R", "T", C)
    got = big.cpu().numpy()
    assert _maxrel(got[10:80], ref) <= 1e-11
    assert not got[:10].any() and not got[80:].any()
    hA, hT, hC = to_host(dA), T.cpu().numpy(), np.asfortranarray(C)
    tqr.tqr_ormqr("R", "T", hA, nb, ib, hT, hC)
    assert np.array_equal(hC, got[10:80])
    hQ = tqr.tqr_orgqr(hA, nb, ib, hT, 150)
    assert np.array_equal(hQ, to_host(tqr.tqr_orgqr(dA, nb, ib, T, 150)))


def test_orgqr_equals_q_applied_to_identity_columns():
    """The skipped steps of the explicit-Q graph touch only exact zeros: its
    columns match Q applied to the same identity columns by the full graph."""
    torch = torch_cuda()
    m, n, nb, ib = 900, 900, 64, 16
    A = inputs.normal_matrix(m, n, 71)
    dA, T, _, _ = _factor(A, nb, ib)
    Q = to_host(tqr.tqr_orgqr(dA, nb, ib, T, m))
    cols = [0, 63, 64, 500, 899]
    E = tqr.colmajor(torch.eye(m, dtype=torch.float64, device="cuda")[:, cols].contiguous())
    tqr.tqr_ormqr("L", "N", dA, nb, ib, T, E)
    assert np.max(np.abs(to_host(E) - Q[:, cols])) <= 4 * U53


def test_empty_and_invalid_arguments():
    torch = torch_cuda()
    m, n, nb, ib = 64, 48, 16, 4
    dA, T, _, _ = _factor(inputs.normal_matrix(m, n, 81), nb, ib)
    assert tqr.tqr_orgqr(dA, nb, ib, T, 0).shape == (m, 0)
    C0 = tqr.colmajor(torch.zeros((0, m), dtype=torch.float64, device="cuda"))
    tqr.tqr_ormqr("R", "N", dA, nb, ib, T, C0)
    bad = tqr.colmajor(torch.zeros((m + 1, 3), dtype=torch.float64, device="cuda"))
    with pytest.raises(tqr.TqrError) as e:
        tqr.tqr_ormqr("L", "N", dA, nb, ib, T, bad)
    assert e.value.code == -11
    with pytest.raises(tqr.TqrError) as e:
        tqr.tqr_ormqr("X", "N", dA, nb, ib, T, bad)
    assert e.value.code == -1
    with pytest.raises(tqr.TqrError) as e:
        tqr.tqr_orgqr(dA, nb, ib, T, m + 1)
    assert e.value.code == -9


def test_full_size_sampled_orgqr():
    """16384 x 16384 N(0,1), nb 128, ib 16 (the benchmark's factorization):
    sampled columns of the explicit Q are orthonormal and reproduce A's
    columns with R."""
    torch = torch_cuda()
    m = n = 16384
    nb, ib = 128, 16
    A = inputs.normal_matrix(m, n, 0)
    dA = to_dev(A)
    T = tqr.tqr_factor(dA, nb, ib)
    Q = tqr.tqr_orgqr(dA, nb, ib, T, n)
    torch.cuda.synchronize()
    cols = [0, 1, 127, 128, 8191, 16383]
    Qs = Q[:, cols].cpu().numpy()
    assert np.linalg.norm(Qs.T @ Qs - np.eye(len(cols))) <= 10 * n * U53
    R = torch.triu(dA)
    for c in cols:
        # A[:, c] = Q[:, :c+1] R[:c+1, c]
        qa = (Q[:, :c + 1] @ R[:c + 1, c]).cpu().numpy()
        assert np.linalg.norm(qa - A[:, c]) / np.linalg.norm(A[:, c]) <= 10 * n * U53
