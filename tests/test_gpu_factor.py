"""GPU parity of the tiled QR against the oracle (called through the C ABI)."""
import numpy as np
import pytest

from oracle import householder as H
from oracle import tiled as TL
from paper_0707_3548_gb300 import inputs, tqr
from tests.gpu_util import t_blocks, to_dev, to_host, torch_cuda

pytestmark = pytest.mark.gpu
U53 = 2.0 ** -53

SHAPES = [
    # m, n, nb, ib  -- several tiles and ragged tails; ib = nb is the paper's kernel
    (512, 512, 128, 32),
    (700, 500, 128, 32),
    (300, 1000, 64, 16),
    (257, 129, 64, 64),
    (600, 400, 192, 64),
    (520, 520, 256, 16),
    (1000, 77, 128, 64),
    (33, 17, 8, 4),
    (1, 1, 8, 8),
    (5, 300, 16, 8),
]


def _factor(A, nb, ib):
    torch_cuda()
    dA = to_dev(A)
    T = tqr.tqr_factor(dA, nb, ib)
    return to_host(dA), T.cpu().numpy()


@pytest.mark.parametrize("m,n,nb,ib", SHAPES)
def test_factor_matches_oracle_elementwise(m, n, nb, ib):
    A = inputs.uniform_matrix(m, n, 17 + m + 3 * n)
    F, Tflat = _factor(A, nb, ib)
    f = TL.tiled_qr(A, nb, ib)
    scale = max(1.0, np.abs(f.F).max())
    assert np.max(np.abs(F - f.F)) <= 1e-11 * scale
    Tg = t_blocks(Tflat, m, n, nb, ib)
    for key, T in f.T.items():
        assert np.max(np.abs(Tg[key] - T)) <= 1e-11 * max(1.0, np.abs(T).max()), key
    # R below the diagonal is exactly zero in the returned R
    R = np.triu(F)
    k = min(m, n)
    Ru = H.sign_normalize(H.r_factor(H.geqr2(A)[0]))[:k]
    assert np.linalg.norm(H.sign_normalize(R)[:k] - Ru) / np.linalg.norm(Ru) <= 1e-11


def test_config1_q_formed():
    """512 x 512, U[-1,1] seed 0, nb 128, ib 32: Q formed; A = QR, Q^T Q = I, R vs oracle."""
    torch = torch_cuda()
    m = n = 512
    A = inputs.uniform_matrix(m, n, 0)
    dA = to_dev(A)
    T = tqr.tqr_factor(dA, 128, 32)
    Q = tqr.colmajor(torch.eye(m, dtype=torch.float64, device="cuda"))
    tqr.tqr_apply_qt("N", dA, 128, 32, T, Q)
    F = to_host(dA)
    Qh = to_host(Q)
    R = np.triu(F)
    tol = 10 * n * U53
    assert np.linalg.norm(A - Qh @ R) / np.linalg.norm(A) <= tol
    assert np.linalg.norm(np.eye(m) - Qh.T @ Qh) <= tol
    Ru = H.sign_normalize(H.r_factor(H.geqr2(A)[0]))
    assert np.linalg.norm(H.sign_normalize(R) - Ru) / np.linalg.norm(Ru) <= 1e-11
    assert np.linalg.norm(R.T @ R - A.T @ A) / np.linalg.norm(A) ** 2 <= tol


@pytest.mark.parametrize("m,n,nb,ib,nrhs", [(700, 500, 128, 32, 3), (300, 600, 64, 16, 40), (256, 256, 64, 64, 1)])
def test_apply_q_and_qt_match_oracle(m, n, nb, ib, nrhs):
    A = inputs.normal_matrix(m, n, 21)
    B = inputs.normal_matrix(m, nrhs, 22)
    dA = to_dev(A)
    T = tqr.tqr_factor(dA, nb, ib)
    f = TL.tiled_qr(A, nb, ib)
    for trans, ref in (("T", TL.apply_qt(f, B)), ("N", TL.apply_q(f, B))):
        dB = to_dev(B)
        tqr.tqr_apply_qt(trans, dA, nb, ib, T, dB)
        assert np.max(np.abs(to_host(dB) - ref)) <= 1e-11 * max(1.0, np.abs(ref).max())


def test_deterministic_across_schedules():
    """Each tile's update sequence is fixed by the DAG, so any schedule gives
    the same bits: repeat, paper priorities, bottom level, 3 CTAs."""
    A = inputs.normal_matrix(900, 700, 5)
    outs = []
    try:
        for policy, cap in ((-1, 0), (-1, 0), (0, 0), (1, 0), (1, 3)):
            tqr.tqr_debug_set_schedule(policy, cap)
            outs.append(_factor(A, 128, 32))
    finally:
        tqr.tqr_debug_set_schedule(-1, 0)
    for F, T in outs[1:]:
        assert np.array_equal(F, outs[0][0]) and np.array_equal(T, outs[0][1])


def test_fp64_bits_do_not_depend_on_the_slab_width():
    """Every FP64 output of an update is one FMA chain over its own column,
    so the slab width (8, 16 or 32 columns per task) changes no bit."""
    A = inputs.normal_matrix(700, 650, 6)
    outs = []
    try:
        for cs in (0, 8, 16, 32):
            tqr.tqr_debug_set_shape(cs, -1)
            outs.append(_factor(A, 64, 16))
    finally:
        tqr.tqr_debug_set_shape(0, -1)
    for F, T in outs[1:]:
        assert np.array_equal(F, outs[0][0]) and np.array_equal(T, outs[0][1])


def test_host_pointer_path_equals_device_path():
    A = inputs.uniform_matrix(300, 200, 8)
    F_dev, T_dev = _factor(A, 64, 16)
    Ah = np.asfortranarray(A.copy())
    Th = tqr.tqr_factor(Ah, 64, 16)
    assert np.array_equal(Ah, F_dev) and np.array_equal(Th, T_dev)


def test_leading_dimension_larger_than_m():
    torch = torch_cuda()
    m, n, lda = 200, 150, 256
    A = inputs.uniform_matrix(m, n, 9)
    big = torch.zeros((n, lda), dtype=torch.float64, device="cuda")
    big[:, :m] = torch.from_numpy(A.T.copy()).cuda()
    view = big.t()[:m, :]            # column-major with lda = 256
    T = tqr.tqr_factor(view, 64, 16)
    F, Tref = _factor(A, 64, 16)
    assert np.array_equal(view.cpu().numpy(), F)
    assert torch.all(big.t()[m:, :] == 0)   # rows past m untouched


def test_empty_and_tiny():
    torch = torch_cuda()
    z = tqr.colmajor(torch.zeros((0, 5), dtype=torch.float64, device="cuda"))
    T = torch.zeros(1, dtype=torch.float64, device="cuda")
    assert tqr.lib().tqr_factor(0, 5, z.data_ptr(), 1, 8, 4, T.data_ptr(), None) == 0
    F, _ = _factor(np.array([[-3.0]]), 8, 8)
    assert F[0, 0] == -3.0   # nothing below alpha: tau = 0, beta = alpha (as the oracle)
    assert TL.tiled_qr(np.array([[-3.0]]), 8, 8).F[0, 0] == -3.0


def test_exact_zero_column_and_padding():
    A = inputs.normal_matrix(70, 40, 11)
    A[:, 5] = 0.0
    A[:, 39] = 0.0
    F, Tflat = _factor(A, 32, 8)
    f = TL.tiled_qr(A, 32, 8)
    assert np.max(np.abs(F - f.F)) <= 1e-11 * np.abs(f.F).max()


def test_bounded_wait_reports_timeout_and_context_survives():
    torch_cuda()
    assert tqr.tqr_debug_stalled_launch(100) == tqr.TQR_ERR_TIMEOUT
    F, _ = _factor(inputs.uniform_matrix(64, 64, 1), 16, 8)
    f = TL.tiled_qr(inputs.uniform_matrix(64, 64, 1), 16, 8)
    assert np.max(np.abs(F - f.F)) <= 1e-12 * np.abs(f.F).max()
    assert tqr.tqr_stream_status() == tqr.TQR_OK


def test_full_size_sampled_parity():
    """8192 x 8192 N(0,1), nb 128, ib 32 (the benchmark's launch): R's leading
    256 x 256 block equals the oracle's QR of A's first 256 columns, and
    Q R reproduces sampled columns of A."""
    torch = torch_cuda()
    m = n = 8192
    A = inputs.normal_matrix(m, n, 0)
    dA = to_dev(A)
    T = tqr.tqr_factor(dA, 128, 32)
    torch.cuda.synchronize()
    lead = dA[:256, :256].cpu().numpy()
    Fo, _ = H.geqr2(A[:, :256])
    assert np.linalg.norm(H.sign_normalize(np.triu(lead)) - H.sign_normalize(np.triu(Fo[:256]))) / \
        np.linalg.norm(Fo[:256]) <= 1e-11
    cols = [0, 1, 127, 128, 4095, 8191]
    Rs = torch.triu(dA)[:, cols].contiguous()
    Rs = tqr.colmajor(Rs)
    tqr.tqr_apply_qt("N", dA, 128, 32, T, Rs)
    err = np.linalg.norm(to_host(Rs) - A[:, cols]) / np.linalg.norm(A[:, cols])
    assert err <= 10 * n * U53


def test_release_cached_memory_then_factor_again():
    """The library's workspace pool can be handed back; later calls allocate
    again and give the same bits."""
    A = inputs.normal_matrix(600, 500, 41)
    F1, T1 = _factor(A, 128, 32)
    tqr.tqr_release_memory()
    F2, T2 = _factor(A, 128, 32)
    assert np.array_equal(F1, F2) and np.array_equal(T1, T2)
    hA = np.array(A, order="F", copy=True)
    hT = tqr.tqr_factor(hA, 128, 32)
    assert np.array_equal(hA, F1)


def test_nonfinite_input_is_reported_by_every_factorization():
    """A NaN or an infinity in A: host-buffer calls return TQR_ERR_NONFINITE,
    device-buffer calls report it through tqr_stream_status (which clears
    it), and a clean call afterwards reports nothing."""
    torch = torch_cuda()
    from paper_0707_3548_gb300.tqr import lib
    A = inputs.normal_matrix(200, 150, 91)
    bad_nan, bad_inf = A.copy(), A.copy()
    bad_nan[17, 33] = np.nan
    bad_inf[199, 149] = -np.inf
    nb, ib = 64, 16
    for bad in (bad_nan, bad_inf):
        # host buffers: the call synchronizes and returns the status
        T = np.zeros(tqr.tqr_t_size(200, 150, nb, ib) // 8)
        h = np.asfortranarray(bad.copy())
        rc = lib().tqr_factor(200, 150, h.ctypes.data, 200, nb, ib, T.ctypes.data, None)
        assert rc == tqr.TQR_ERR_NONFINITE
        # device buffers: asynchronous, reported by tqr_stream_status
        calls = [
            lambda d: tqr.tqr_factor(d, nb, ib, check=False),
            lambda d: tqr.tqr_factor_pairs(d, nb, ib),
            lambda d: tqr.tqr_factor_tree(d, nb, ib, 2),
            lambda d: tqr.tqr_lu_factor(d, nb, ib),
        ]
        for call in calls:
            call(to_dev(bad))
            assert tqr.tqr_stream_status() == tqr.TQR_ERR_NONFINITE
            assert tqr.tqr_stream_status() == tqr.TQR_OK          # cleared
        dA = to_dev(bad)
        Tn = torch.zeros(tqr.tqr_t_size(200, 150, nb, ib) // 8, dtype=torch.float64, device="cuda")
        assert tqr.tqr_factor_noalloc(dA, nb, ib, Tn, check=False) == tqr.TQR_OK
        assert tqr.tqr_stream_status() == tqr.TQR_ERR_NONFINITE
    tqr.tqr_factor(to_dev(A), nb, ib)
    assert tqr.tqr_stream_status() == tqr.TQR_OK
