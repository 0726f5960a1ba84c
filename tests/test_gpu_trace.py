"""The device task trace (tqr_debug_trace): every task of Algorithm 1 runs
exactly once, and no task starts before the tasks it depends on (Section 3.2's
DAG: GEQRT(k) after SSRFB(k-1,k,k); LARFB(k,j) after GEQRT(k) and
SSRFB(k-1,k,j); TSQRT(k,i) after TSQRT(k,i-1) (GEQRT(k) for i = k+1) and
SSRFB(k-1,i,k); SSRFB(k,i,j) after TSQRT(k,i), the previous writer of (k,j)
and SSRFB(k-1,i,j)) have finished, checked on the timestamps the kernel
wrote.  Tracing changes no result."""
import numpy as np
import pytest

from paper_0707_3548_gb300 import inputs, tqr
from tests.gpu_util import to_dev, to_host, torch_cuda

pytestmark = pytest.mark.gpu
GEQRT, TSQRT, LARFB, SSRFB = 0, 1, 2, 3


def _traced_factor(A, nb, ib, cap, extra=0):
    torch = torch_cuda()
    buf = torch.zeros((cap + extra, 8), dtype=torch.int64, device="cuda")
    dA = to_dev(A)
    tqr.tqr_debug_trace(buf[:cap])
    try:
        T = tqr.tqr_factor(dA, nb, ib)
        torch.cuda.synchronize()
    finally:
        tqr.tqr_debug_trace(None)
    return to_host(dA), T.cpu().numpy(), buf.cpu().numpy()


@pytest.mark.parametrize("m,n,nb,ib", [(1024, 768, 64, 16), (700, 900, 128, 32)])
def test_trace_covers_algorithm_1_and_respects_the_dag(m, n, nb, ib):
    A = inputs.normal_matrix(m, n, 7)
    F, T, words = _traced_factor(A, nb, ib, 20000)
    dA = to_dev(A)
    T2 = tqr.tqr_factor(dA, nb, ib)
    assert np.array_equal(F, to_host(dA)) and np.array_equal(T, T2.cpu().numpy())

    r = tqr.trace_records(words)
    assert len(tqr.trace_chrome(words)["traceEvents"]) == len(r["kind"])
    p, q = -(-m // nb), -(-n // nb)
    kt = min(p, q)
    assert np.all(r["ticket_ns"] <= r["start_ns"]) and np.all(r["start_ns"] <= r["end_ns"])
    start, end = {}, {}
    for a in range(len(r["kind"])):
        key = (int(r["kind"][a]), int(r["k"][a]), int(r["i"][a]), int(r["j"][a]), int(r["s"][a]))
        assert key not in start, key
        start[key], end[key] = int(r["start_ns"][a]), int(r["end_ns"][a])
    slabs = sorted({key[4] for key in start if key[0] == LARFB})
    assert slabs == list(range(len(slabs))) and nb % len(slabs) == 0
    S = range(len(slabs))
    expected = set()
    for k in range(kt):
        expected.add((GEQRT, k, k, k, 0))
        expected |= {(TSQRT, k, i, k, 0) for i in range(k + 1, p)}
        expected |= {(LARFB, k, k, j, s) for j in range(k + 1, q) for s in S}
        expected |= {(SSRFB, k, i, j, s) for i in range(k + 1, p) for j in range(k + 1, q) for s in S}
    assert set(start) == expected

    def after(task, dep):
        if dep in end:
            assert end[dep] <= start[task], (task, dep)

    for (kind, k, i, j, s) in start:
        t = (kind, k, i, j, s)
        if kind == GEQRT and k > 0:
            for s2 in S:
                after(t, (SSRFB, k - 1, k, k, s2))
        elif kind == LARFB:
            after(t, (GEQRT, k, k, k, 0))
            if k > 0:
                after(t, (SSRFB, k - 1, k, j, s))
        elif kind == TSQRT:
            after(t, (GEQRT, k, k, k, 0) if i == k + 1 else (TSQRT, k, i - 1, k, 0))
            if k > 0:
                for s2 in S:
                    after(t, (SSRFB, k - 1, i, k, s2))
        elif kind == SSRFB:
            after(t, (TSQRT, k, i, k, 0))
            after(t, (LARFB, k, k, j, s) if i == k + 1 else (SSRFB, k, i - 1, j, s))
            if k > 0:
                after(t, (SSRFB, k - 1, i, j, s))


def test_trace_stops_at_its_capacity():
    A = inputs.normal_matrix(512, 512, 8)
    _, _, words = _traced_factor(A, 64, 16, 50, extra=64)
    assert np.all(words[:50, 2] != 0)
    assert not words[50:].any()
