"""Least-squares server: continuous batching over concurrent requests with
resident factorizations.  Each request's result must be the same alone and in
the mix, and match the oracle."""
import numpy as np
import pytest

from oracle import lstsq as LS
from paper_0707_3548_gb300 import inputs, tqr
from tests.gpu_util import to_dev, to_host, torch_cuda

pytestmark = pytest.mark.gpu


def _workload(seed=5, count=24):
    g = inputs.rng(seed)
    mats = []
    reqs = []
    for r in range(count):
        if mats and g.uniform() < 0.3:
            mid = int(g.integers(0, len(mats)))
        else:
            m = int(g.integers(128, 900))
            n = int(g.integers(64, max(65, m // 2)))
            mats.append(inputs.normal_matrix(m, n, 1000 + len(mats)))
            mid = len(mats) - 1
        nrhs = int(g.integers(1, 17))
        prec = tqr.TQR_PREC_FP32 if r % 2 else tqr.TQR_PREC_FP64
        B = inputs.normal_matrix(mats[mid].shape[0], nrhs, 5000 + r)
        reqs.append((mid, B, prec))
    return mats, reqs


def _run(server, dmats, reqs, one_at_a_time):
    torch = torch_cuda()
    outs, infos, ids = [], [], []
    for mid, B, prec in reqs:
        dB = to_dev(B)
        X = tqr.colmajor(torch.zeros((dmats[mid].shape[1], B.shape[1]), dtype=torch.float64, device="cuda"))
        rid = server.submit(mid, dmats[mid], dB, X, prec=prec)
        outs.append((X, dB))
        ids.append(rid)
        if one_at_a_time:
            infos.append(server.wait(rid))
    if not one_at_a_time:
        infos = [server.wait(r) for r in ids]
    return [to_host(X) for X, _ in outs], infos


def test_server_results_same_alone_and_in_the_mix():
    torch_cuda()
    mats, reqs = _workload()
    dmats = [to_dev(A) for A in mats]
    mix_server = tqr.Server(4 << 30, slots=4)
    try:
        X_mix, info_mix = _run(mix_server, dmats, reqs, one_at_a_time=False)
        stats = mix_server.stats()
    finally:
        mix_server.close()
    alone_server = tqr.Server(4 << 30, slots=4)
    try:
        X_alone, info_alone = _run(alone_server, dmats, reqs, one_at_a_time=True)
    finally:
        alone_server.close()
    bad = [(k, i["status"], i["iters"], i["berr"]) for k, i in enumerate(info_mix + info_alone) if i["status"] != 0]
    assert stats["completed"] == len(reqs) and stats["failed"] == 0, bad
    assert stats["reused"] == sum(i["reused"] for i in info_mix) > 0
    for (mid, B, prec), xm, xa, im, ia in zip(reqs, X_mix, X_alone, info_mix, info_alone):
        assert im["status"] == 0 and ia["status"] == 0
        assert im["berr"] <= 1e-12
        assert np.array_equal(xm, xa), (mid, prec)
        xo = LS.lstsq(mats[mid], B)
        assert np.max(np.abs(xm - xo)) <= 1e-10 * max(1.0, np.abs(xo).max())


def test_server_budget_eviction_keeps_working():
    torch = torch_cuda()
    A = [inputs.normal_matrix(600, 200, 70 + a) for a in range(6)]
    dA = [to_dev(x) for x in A]
    s = tqr.Server(24 << 20, slots=2)   # room for about one resident factorization
    try:
        for rep in range(2):
            for a in range(6):
                B = inputs.normal_matrix(600, 3, 80 + a)
                X = tqr.colmajor(torch.zeros((200, 3), dtype=torch.float64, device="cuda"))
                info = s.wait(s.submit(a, dA[a], to_dev(B), X))
                assert info["status"] == 0
                assert np.allclose(to_host(X), LS.lstsq(A[a], B), atol=1e-10)
        st = s.stats()
        assert st["bytes_in_use"] <= 24 << 20
    finally:
        s.close()


def test_request_larger_than_the_budget_is_refused():
    """A request whose workspace exceeds the whole HBM budget finishes with
    TQR_ERR_NOMEM instead of waiting for room; a request that fits still runs."""
    import time

    torch = torch_cuda()
    s = tqr.Server(16 << 20, slots=1)
    try:
        big = inputs.normal_matrix(3000, 1000, 90)          # 24 MB of A alone
        Xb = tqr.colmajor(torch.zeros((1000, 1), dtype=torch.float64, device="cuda"))
        rid = s.submit(0, to_dev(big), to_dev(inputs.normal_matrix(3000, 1, 91)), Xb)
        info, deadline = None, time.time() + 60
        while info is None and time.time() < deadline:
            info = s.poll(rid)
            time.sleep(0.01)
        assert info is not None and info["status"] == tqr.TQR_ERR_NOMEM
        why = s.last_failure()
        assert "3000 x 1000" in why and "status %d" % tqr.TQR_ERR_NOMEM in why, why
        A = inputs.normal_matrix(300, 100, 92)
        B = inputs.normal_matrix(300, 2, 93)
        X = tqr.colmajor(torch.zeros((100, 2), dtype=torch.float64, device="cuda"))
        info = s.wait(s.submit(1, to_dev(A), to_dev(B), X))
        assert info["status"] == 0
        assert np.allclose(to_host(X), LS.lstsq(A, B), atol=1e-10)
    finally:
        s.close()
