"""GPU parity of the tiled LU with pairwise pivoting (tqr_lu_factor /
tqr_lu_solve through the C ABI) against the oracle."""
import numpy as np
import pytest

from oracle import tiled_lu as LU
from paper_0707_3548_gb300 import inputs, tqr
from tests.gpu_util import to_dev, to_host, torch_cuda

pytestmark = pytest.mark.gpu
U53 = 2.0 ** -53


def _slots(m, n, nb):
    p, q = -(-m // nb), -(-n // nb)
    return [(i, k) for k in range(min(p, q)) for i in range(k, p)]


def _factor(A, nb, ib):
    torch_cuda()
    dA = to_dev(A)
    L, piv = tqr.tqr_lu_factor(dA, nb, ib)
    return dA, L, piv


SHAPES = [
    # m, n, nb, ib -- several tiles, ragged tails, rectangular, ib = nb
    (512, 512, 128, 32),
    (700, 500, 128, 32),
    (300, 600, 64, 16),
    (257, 257, 64, 64),
    (1000, 1000, 128, 16),
    (33, 17, 8, 4),
    (5, 300, 16, 8),
]


@pytest.mark.parametrize("m,n,nb,ib", SHAPES)
def test_lu_factor_matches_oracle(m, n, nb, ib):
    A = inputs.normal_matrix(m, n, 101 + m + n)
    dA, L, piv = _factor(A, nb, ib)
    f = LU.tiled_lu(A, nb, ib)
    F = to_host(dA)
    ref = f.Ap[:m, :n]
    assert np.max(np.abs(F - ref)) <= 1e-10 * max(1.0, np.abs(ref).max())
    pv = piv.cpu().numpy()
    Lh = L.cpu().numpy()
    for idx, (i, k) in enumerate(_slots(m, n, nb)):
        got = pv[idx * nb:(idx + 1) * nb]
        assert np.array_equal(got, f.piv[(i, k)]), (i, k)
        # L holds, per ib block, the inverse of the block's unit lower triangle (transposed)
        blocks = Lh[idx * ib * nb:(idx + 1) * ib * nb].reshape(nb, ib).T     # ib x nb, column-major
        for l0 in range(0, nb, ib):
            if i == k:
                L11 = np.tril(f.tile(k, k)[l0:l0 + ib, l0:l0 + ib], -1) + np.eye(ib)
            else:
                L11 = np.tril(f.L1[(i, k)][:, l0:l0 + ib], -1) + np.eye(ib)
            X = np.linalg.inv(L11)
            assert np.max(np.abs(blocks[:, l0:l0 + ib].T - X)) <= 1e-10 * max(1.0, np.abs(X).max())


@pytest.mark.parametrize("n,nb,ib,nrhs", [(512, 128, 32, 3), (700, 64, 16, 40), (257, 64, 64, 1), (33, 8, 4, 5)])
def test_lu_solve_matches_oracle(n, nb, ib, nrhs):
    A = inputs.normal_matrix(n, n, 111 + n)
    B = inputs.normal_matrix(n, nrhs, 112)
    dA, L, piv = _factor(A, nb, ib)
    dB = to_dev(B)
    tqr.tqr_lu_solve(dA, nb, ib, L, piv, dB)
    X = to_host(dB)
    f = LU.tiled_lu(A, nb, ib)
    ref = LU.lu_solve(f, B)
    # same pivots, both backward stable: the solutions differ by about kappa * (n u)
    assert np.max(np.abs(X - ref)) <= 1e-12 * np.linalg.cond(A) * max(1.0, np.abs(ref).max())
    assert np.linalg.norm(A @ X - B) / (np.linalg.norm(A) * np.linalg.norm(X)) <= 1e3 * n * U53


def test_deterministic_across_schedules():
    A = inputs.normal_matrix(900, 900, 7)
    outs = []
    try:
        for policy, cap in ((-1, 0), (-1, 0), (0, 0), (1, 0), (1, 3)):
            tqr.tqr_debug_set_schedule(policy, cap)
            dA, L, piv = _factor(A, 128, 32)
            outs.append((to_host(dA), L.cpu().numpy(), piv.cpu().numpy()))
    finally:
        tqr.tqr_debug_set_schedule(-1, 0)
    for o in outs[1:]:
        assert all(np.array_equal(a, b) for a, b in zip(o, outs[0]))


def test_host_pointer_path_equals_device_path():
    A = inputs.normal_matrix(300, 300, 9)
    B = inputs.normal_matrix(300, 4, 10)
    dA, L, piv = _factor(A, 64, 16)
    hA = np.array(A, order="F", copy=True)
    hL, hp = tqr.tqr_lu_factor(hA, 64, 16)
    assert np.array_equal(hA, to_host(dA)) and np.array_equal(hL, L.cpu().numpy()) and \
        np.array_equal(hp, piv.cpu().numpy())
    hB = np.array(B, order="F", copy=True)
    tqr.tqr_lu_solve(hA, 64, 16, hL, hp, hB)
    dB = to_dev(B)
    tqr.tqr_lu_solve(dA, 64, 16, L, piv, dB)
    assert np.array_equal(hB, to_host(dB))


def test_zero_diagonal_tile_pivots_from_below():
    """A_00 = 0: GETRF meets zero pivots and leaves them; TSTRF takes every
    pivot from the tile below."""
    nb = 16
    Z = np.zeros((nb, nb))
    Q = inputs.normal_matrix(nb, nb, 11) + 4 * np.eye(nb)
    A = np.block([[Z, np.eye(nb)], [Q, inputs.normal_matrix(nb, nb, 12)]])
    dA, L, piv = _factor(A, nb, 4)
    f = LU.tiled_lu(A, nb, 4)
    assert np.max(np.abs(to_host(dA) - f.Ap)) <= 1e-12 * np.abs(f.Ap).max()
    pv = piv.cpu().numpy()
    assert (pv[nb:2 * nb] >= 0).all()          # slot (1, 0): every column swapped with the bottom tile
    B = inputs.normal_matrix(2 * nb, 2, 13)
    dB = to_dev(B)
    tqr.tqr_lu_solve(dA, nb, 4, L, piv, dB)
    assert np.linalg.norm(A @ to_host(dB) - B) <= 1e-11 * np.linalg.norm(B) * np.linalg.cond(A)


def test_invalid_arguments():
    torch = torch_cuda()
    A = to_dev(inputs.normal_matrix(64, 64, 14))
    with pytest.raises(tqr.TqrError) as e:
        tqr.tqr_lu_factor(A, 16, 5)
    assert e.value.code == -6
    L, piv = tqr.tqr_lu_factor(A, 16, 4)
    bad = tqr.colmajor(torch.zeros((60, 2), dtype=torch.float64, device="cuda"))
    with pytest.raises(tqr.TqrError) as e:
        tqr.tqr_lu_solve(A, 16, 4, L, piv, bad)
    assert e.value.code == -10


def test_full_size_sampled_lu():
    """16384 x 16384 N(0,1), nb 128, ib 16 (the benchmark's launch): the
    first diagonal tile equals the oracle's GETRF of A's leading tile, and a
    solve through the factors has a small backward error."""
    torch = torch_cuda()
    n, nb, ib = 16384, 128, 16
    A = inputs.normal_matrix(n, n, 0)
    dA0 = to_dev(A)
    dA = dA0.clone()
    dA = tqr.colmajor(dA)
    L, piv = tqr.tqr_lu_factor(dA, nb, ib)
    torch.cuda.synchronize()
    F00, p00 = LU.getrf(A[:nb, :nb], ib)
    # tile (0, 0) is final after its TSTRFs only in its strictly lower part
    got = dA[:nb, :nb].cpu().numpy()
    assert np.max(np.abs(np.tril(got, -1) - np.tril(F00, -1))) <= 1e-10 * np.abs(F00).max()
    assert np.array_equal(piv[:nb].cpu().numpy(), p00)
    x = torch.from_numpy(inputs.normal_matrix(n, 1, 1)).cuda()
    b = tqr.colmajor(dA0 @ x)
    r0 = b.clone()
    tqr.tqr_lu_solve(dA, nb, ib, L, piv, b)
    res = torch.linalg.norm(dA0 @ b - r0).item()
    assert res / (torch.linalg.norm(dA0).item() * torch.linalg.norm(b).item()) <= 1e3 * n * U53


# 2b x b bottoms -------------------------------------------------------------

@pytest.mark.parametrize("m,n,nb,ib", [(512, 512, 128, 32), (700, 500, 128, 32), (1000, 1000, 128, 16),
                                       (300, 600, 64, 16), (33, 17, 8, 4)])
def test_lu_pairs_match_oracle(m, n, nb, ib):
    torch_cuda()
    A = inputs.normal_matrix(m, n, 301 + m + n)
    dA = to_dev(A)
    L, piv = tqr.tqr_lu_factor(dA, nb, ib, pairs=True)
    f = LU.tiled_lu_pairs(A, nb, ib)
    ref = f.Ap[:m, :n]
    assert np.max(np.abs(to_host(dA) - ref)) <= 1e-10 * max(1.0, np.abs(ref).max())
    pv = piv.cpu().numpy()
    slots = _slots(m, n, nb)
    for key, p_ref in f.piv.items():
        idx = slots.index(key)
        assert np.array_equal(pv[idx * nb:(idx + 1) * nb], p_ref), key


@pytest.mark.parametrize("n,nb,ib,nrhs", [(512, 128, 32, 3), (700, 64, 16, 40)])
def test_lu_pairs_solve(n, nb, ib, nrhs):
    A = inputs.normal_matrix(n, n, 311 + n)
    B = inputs.normal_matrix(n, nrhs, 312)
    dA = to_dev(A)
    L, piv = tqr.tqr_lu_factor(dA, nb, ib, pairs=True)
    dB = to_dev(B)
    tqr.tqr_lu_solve(dA, nb, ib, L, piv, dB, pairs=True)
    X = to_host(dB)
    ref = LU.pairs_lu_solve(LU.tiled_lu_pairs(A, nb, ib), B)
    assert np.max(np.abs(X - ref)) <= 1e-12 * np.linalg.cond(A) * max(1.0, np.abs(ref).max())
    assert np.linalg.norm(A @ X - B) / (np.linalg.norm(A) * np.linalg.norm(X)) <= 1e3 * n * U53


def test_lu_pairs_host_path_and_plan_separation():
    A = inputs.normal_matrix(400, 400, 313)
    dA = to_dev(A)
    L, piv = tqr.tqr_lu_factor(dA, 64, 16, pairs=True)
    hA = np.array(A, order="F", copy=True)
    hL, hp = tqr.tqr_lu_factor(hA, 64, 16, pairs=True)
    assert np.array_equal(hA, to_host(dA)) and np.array_equal(hp, piv.cpu().numpy())
    # the flat LU of the same shape right after must run its own task list
    dA2 = to_dev(A)
    tqr.tqr_lu_factor(dA2, 64, 16)
    f = LU.tiled_lu(A, 64, 16)
    assert np.max(np.abs(to_host(dA2) - f.Ap[:400, :400])) <= 1e-10 * np.abs(f.Ap).max()


@pytest.mark.parametrize("m,n,nb,ib", [(1, 1, 8, 8), (5, 3, 8, 4), (8, 8, 8, 2), (17, 40, 8, 4), (24, 1, 8, 8),
                                       (40, 17, 8, 8)])
@pytest.mark.parametrize("pairs", [False, True])
def test_lu_tiny_and_degenerate_shapes(m, n, nb, ib, pairs):
    torch_cuda()
    A = inputs.uniform_matrix(m, n, 321 + m + n)
    dA = to_dev(A)
    tqr.tqr_lu_factor(dA, nb, ib, pairs=pairs)
    f = LU.tiled_lu_pairs(A, nb, ib) if pairs else LU.tiled_lu(A, nb, ib)
    assert np.max(np.abs(to_host(dA) - f.Ap[:m, :n])) <= 1e-11 * max(1.0, np.abs(f.Ap).max())
