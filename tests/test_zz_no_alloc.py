"""tqr_factor_noalloc, the factorization for callers that cannot allocate
device memory (a process whose HBM was all handed to another allocator at
start-up, or code that may not risk an allocation's latency or failure).  Its
scratch is a static device array inside libtqr.

The checks call the new entry point through the C ABI and compare it with
tqr_factor over calls in a row (the array keeps the previous call's contents,
so stale counters would show).  Each tile's sequence of updates is fixed by
the task DAG, so the sequential task order of this entry point and the
scheduled order of tqr_factor give the same bits: F and T must be equal.
The file name makes pytest collect it last, so a run that stops at the first
failure has already run every other test; it also passes on its own in a
fresh process."""
import numpy as np
import pytest

from paper_0707_3548_gb300 import inputs, tqr
from tests.gpu_util import to_dev, to_host, torch_cuda

pytestmark = pytest.mark.gpu


def _reference(A, nb, ib):
    dA = to_dev(A)
    T = tqr.tqr_factor(dA, nb, ib)
    return to_host(dA), T.cpu().numpy()


def _noalloc(A, nb, ib):
    torch = torch_cuda()
    dA = to_dev(A)
    cnt = tqr.tqr_t_size(A.shape[0], A.shape[1], nb, ib) // 8
    T = torch.full((cnt,), float("nan"), dtype=torch.float64, device="cuda")
    rc = tqr.tqr_factor_noalloc(dA, nb, ib, T, check=False)
    torch.cuda.synchronize()
    return rc, to_host(dA), T.cpu().numpy()


def test_noalloc_matches_tqr_factor_on_calls_in_a_row():
    torch_cuda()
    cases = [(700, 500, 128, 32, 1), (700, 500, 128, 32, 2), (300, 1000, 64, 16, 3), (129, 65, 32, 32, 4)]
    for m, n, nb, ib, seed in cases:
        A = inputs.normal_matrix(m, n, seed)
        rc, F, T = _noalloc(A, nb, ib)
        assert rc == tqr.TQR_OK
        assert tqr.tqr_stream_status() == tqr.TQR_OK
        Fr, Tr = _reference(A, nb, ib)
        assert np.array_equal(F, Fr), (m, n, seed, np.max(np.abs(F - Fr)))
        assert np.array_equal(T, Tr), (m, n, seed, np.max(np.abs(T - Tr)))


def test_noalloc_rejects_what_does_not_fit():
    torch = torch_cuda()
    A = tqr.colmajor(torch.zeros((8, 8), dtype=torch.float64, device="cuda"))
    T = torch.zeros(64, dtype=torch.float64, device="cuda")
    # 4096 x 4096 padded tiles need 16 Mi doubles, above the static maximum
    rc = tqr.lib().tqr_factor_noalloc(4096, 4096, A.data_ptr(), 4096, 128, 32, T.data_ptr(), None)
    assert rc == tqr.TQR_ERR_TOO_LARGE
    # host buffers would need staging memory: rejected as an invalid argument
    h = np.zeros((8, 8), order="F")
    rc = tqr.lib().tqr_factor_noalloc(8, 8, h.ctypes.data, 8, 8, 4, T.data_ptr(), None)
    assert rc == -3
