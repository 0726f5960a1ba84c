"""Batched factorization: one persistent launch over many independent matrices."""
import numpy as np
import pytest

from oracle import tiled as TL
from paper_0707_3548_gb300 import inputs, tqr
from tests.gpu_util import to_dev, to_host, torch_cuda

pytestmark = pytest.mark.gpu


def _alone(A, nb, ib):
    dA = to_dev(A)
    T = tqr.tqr_factor(dA, nb, ib)
    return to_host(dA), T.cpu().numpy()


def _submit(mats, tiles):
    torch = torch_cuda()
    dev = [to_dev(A) for A in mats]
    Ts = []
    for A, (nb, ib) in zip(mats, tiles):
        Ts.append(torch.zeros(tqr.tqr_t_size(A.shape[0], A.shape[1], nb, ib) // 8, dtype=torch.float64,
                              device="cuda"))
    t = tqr.tqr_batch_submit(dev, Ts, tiles)
    return t, dev, Ts


def test_batch_equals_factoring_each_alone():
    torch_cuda()
    shapes = inputs.batch_shapes(40, seed=3, m_lo=16, m_hi=700, n_lo=4)
    mats = inputs.batch_matrices(shapes, seed=3)
    tiles = [tqr.tqr_autotune(m, n) for m, n in shapes]
    t, dev, Ts = _submit(mats, tiles)
    rc, st = tqr.tqr_batch_wait(t, len(mats))
    assert rc == 0 and not st.any()
    for A, dA, T, (nb, ib) in zip(mats, dev, Ts, tiles):
        F, Tr = _alone(A, nb, ib)
        assert np.array_equal(to_host(dA), F)
        assert np.array_equal(T.cpu().numpy(), Tr)
    # a few against the oracle directly
    for A, dA, (nb, ib) in list(zip(mats, dev, tiles))[:5]:
        f = TL.tiled_qr(A, nb, ib)
        assert np.max(np.abs(to_host(dA) - f.F)) <= 1e-11 * max(1.0, np.abs(f.F).max())



def test_pairs_batch_equals_factor_pairs_alone():
    """tqr_batch_submit_pairs: every matrix as tqr_factor_pairs alone (same
    bits, A and T), ragged shapes with odd and even tile-row counts, plus a
    few against the 2b x b oracle."""
    torch = torch_cuda()
    shapes = inputs.batch_shapes(30, seed=5, m_lo=16, m_hi=900, n_lo=4)
    mats = inputs.batch_matrices(shapes, seed=5)
    tiles = [tqr.tqr_autotune(m, n) for m, n in shapes]
    dev = [to_dev(A) for A in mats]
    Ts = [torch.zeros(tqr.tqr_t_size(m, n, nb, ib) // 8, dtype=torch.float64, device="cuda")
          for (m, n), (nb, ib) in zip(shapes, tiles)]
    t = tqr.tqr_batch_submit(dev, Ts, tiles, pairs=True)
    rc, st = tqr.tqr_batch_wait(t, len(mats))
    assert rc == 0 and not st.any()
    for A, dA, T, (nb, ib) in zip(mats, dev, Ts, tiles):
        dB = to_dev(A)
        Tr = tqr.tqr_factor_pairs(dB, nb, ib)
        assert np.array_equal(to_host(dA), to_host(dB))
        assert np.array_equal(T.cpu().numpy(), Tr.cpu().numpy())
    for A, dA, (nb, ib) in list(zip(mats, dev, tiles))[:4]:
        f = TL.tiled_qr_pairs(A, nb, ib)
        assert np.max(np.abs(to_host(dA) - f.F)) <= 1e-11 * max(1.0, np.abs(f.F).max())


def test_batch_reports_nonfinite_per_matrix():
    """A NaN in one matrix and an infinity in another: those two report
    TQR_ERR_NONFINITE, the batch returns it, and every other matrix is
    factored exactly as alone; a resubmission of the same shapes with finite
    data (the graph replay) reports all clear."""
    torch_cuda()
    shapes = [(200, 120), (64, 64), (333, 17), (90, 90), (150, 150)]
    tiles = [(64, 16), (32, 8), (32, 16), (32, 8), (64, 16)]
    mats = [inputs.normal_matrix(m, n, 40 + a) for a, (m, n) in enumerate(shapes)]
    mats[1][5, 7] = np.nan
    mats[3][80, 2] = np.inf
    t, dev, Ts = _submit(mats, tiles)
    rc, st = tqr.tqr_batch_wait(t, len(mats))
    assert rc == tqr.TQR_ERR_NONFINITE
    assert list(st) == [0, tqr.TQR_ERR_NONFINITE, 0, tqr.TQR_ERR_NONFINITE, 0]
    for a in (0, 2, 4):
        F, Tr = _alone(mats[a], *tiles[a])
        assert np.array_equal(to_host(dev[a]), F)
        assert np.array_equal(Ts[a].cpu().numpy(), Tr)
    clean = [inputs.normal_matrix(m, n, 60 + a) for a, (m, n) in enumerate(shapes)]
    t, dev, Ts = _submit(clean, tiles)
    rc, st = tqr.tqr_batch_wait(t, len(clean))
    assert rc == 0 and not st.any()


def test_unpolled_ticket_keeps_its_statuses_when_the_plan_is_reused():
    """A finished batch that was never polled, then a new submission of the
    same shapes: the first ticket still reports its own per-matrix statuses
    (here a NaN in matrix 2), the second its own."""
    torch = torch_cuda()
    shapes = [(120, 80), (77, 77), (210, 40)]
    tiles = [(32, 8), (32, 8), (64, 16)]
    first = [inputs.normal_matrix(m, n, 70 + a) for a, (m, n) in enumerate(shapes)]
    first[2][3, 3] = np.nan
    t1, dev1, Ts1 = _submit(first, tiles)
    torch.cuda.synchronize()
    second = [inputs.normal_matrix(m, n, 80 + a) for a, (m, n) in enumerate(shapes)]
    t2, dev2, Ts2 = _submit(second, tiles)
    rc2, st2 = tqr.tqr_batch_wait(t2, len(second))
    rc1, st1 = tqr.tqr_batch_wait(t1, len(first))
    assert rc1 == tqr.TQR_ERR_NONFINITE and list(st1) == [0, 0, tqr.TQR_ERR_NONFINITE]
    assert rc2 == 0 and not st2.any()
    for a in range(len(second)):
        F, Tr = _alone(second[a], *tiles[a])
        assert np.array_equal(to_host(dev2[a]), F)

def test_batch_graph_replay_with_new_data_and_poll():
    torch = torch_cuda()
    shapes = [(200, 120), (64, 64), (333, 17), (90, 90)]
    tiles = [(64, 16), (32, 8), (32, 16), (48, 16)]
    for seed in (11, 12):      # second submission replays the captured graph
        mats = [inputs.normal_matrix(m, n, seed * 100 + a) for a, (m, n) in enumerate(shapes)]
        t, dev, Ts = _submit(mats, tiles)
        done = False
        for _ in range(100000):
            done, rc, st = tqr.tqr_batch_poll(t, len(mats))
            if done:
                break
        if not done:
            rc, st = tqr.tqr_batch_wait(t, len(mats))
        assert rc == 0 and not st.any()
        for A, dA, (nb, ib) in zip(mats, dev, tiles):
            F, _ = _alone(A, nb, ib)
            assert np.array_equal(to_host(dA), F)
    assert tqr.lib().tqr_batch_poll(987654321, tqr.ctypes.byref(tqr.ctypes.c_int(0)), None) == -1


def test_measured_autotuner_picks_a_candidate_and_the_batch_uses_it(tmp_path):
    """tqr_autotune_run times the candidates of one size class on the device
    and stores the winner; tqr_autotune and a batch with the library's
    choice then use it, and the factors equal those of factoring each
    matrix alone with that (nb, ib) and the oracle's."""
    torch_cuda()
    tqr.tqr_autotune_clear()
    try:
        tqr.tqr_autotune_run(300, 200)
        nb, ib = tqr.tqr_autotune(300, 200)
        assert nb in (16, 32, 64, 96, 128, 192, 256) and ib in (8, 16, 32) and nb % ib == 0
        assert tqr.tqr_autotune(257, 129) == (nb, ib)          # same class (9, 8)
        path = tmp_path / "tune.txt"
        tqr.tqr_autotune_save(str(path))
        assert ("9 8 %d %d" % (nb, ib)) in path.read_text()
        shapes = [(300, 200), (280, 150), (257, 256)]
        mats = [inputs.normal_matrix(m, n, 80 + a) for a, (m, n) in enumerate(shapes)]
        tiles = [tqr.tqr_autotune(m, n) for m, n in shapes]
        assert all(t == (nb, ib) for t in tiles)
        t, dev, Ts = _submit(mats, tiles)
        rc, st = tqr.tqr_batch_wait(t, len(mats))
        assert rc == 0 and not st.any()
        for A, dA in zip(mats, dev):
            F, _ = _alone(A, nb, ib)
            assert np.array_equal(to_host(dA), F)
            f = TL.tiled_qr(A, nb, ib)
            assert np.max(np.abs(F - f.F)) <= 1e-11 * np.abs(f.F).max()
    finally:
        tqr.tqr_autotune_clear()


def test_batch_policy_tuner_writes_one_choice_per_class_and_the_batch_is_correct():
    """tqr_autotune_batch measures the classes of a batch and five tile
    policies on the batch's own shapes, then stores one (nb, ib) per class;
    the batch factored with the library's choice matches factoring each
    matrix alone and the oracle."""
    torch_cuda()
    tqr.tqr_autotune_clear()
    try:
        shapes = inputs.batch_shapes(24, seed=11, m_lo=40, m_hi=300, n_lo=8)
        tqr.tqr_autotune_batch(shapes)
        tiles = [tqr.tqr_autotune(m, n) for m, n in shapes]
        by_class = {}
        for (m, n), t in zip(shapes, tiles):
            by_class.setdefault(tqr.tqr_debug_autotune_class(m, n), set()).add(t)
        assert all(len(v) == 1 for v in by_class.values())
        for nb, ib in tiles:
            assert nb % 8 == 0 and nb % ib == 0
        mats = inputs.batch_matrices(shapes, seed=11)
        t, dev, Ts = _submit(mats, tiles)
        rc, st = tqr.tqr_batch_wait(t, len(mats))
        assert rc == 0 and not st.any()
        for A, dA, (nb, ib) in zip(mats, dev, tiles):
            F, _ = _alone(A, nb, ib)
            assert np.array_equal(to_host(dA), F)
            f = TL.tiled_qr(A, nb, ib)
            assert np.max(np.abs(F - f.F)) <= 1e-11 * np.abs(f.F).max()
    finally:
        tqr.tqr_autotune_clear()


def test_batch_with_config_sized_matrices_up_to_2048():
    """Matrices of the batch benchmark's size range (m up to 2048, n up to m)
    in one launch with the library's tile choice: each equals factoring it
    alone, and its R satisfies R^T R = A^T A to 10 n u of ||A||_F^2 (a
    backward-stable factorization's bound, independent of conditioning)."""
    torch_cuda()
    shapes = [(2048, 2048), (2048, 1500), (1900, 37), (1024, 1024), (777, 500), (64, 32), (1300, 1299)]
    mats = [inputs.normal_matrix(m, n, 300 + a) for a, (m, n) in enumerate(shapes)]
    tiles = [tqr.tqr_autotune(m, n) for m, n in shapes]
    t, dev, Ts = _submit(mats, tiles)
    rc, st = tqr.tqr_batch_wait(t, len(mats))
    assert rc == 0 and not st.any()
    for A, dA, (nb, ib) in zip(mats, dev, tiles):
        F = to_host(dA)
        Fa, _ = _alone(A, nb, ib)
        assert np.array_equal(F, Fa)
        k = min(A.shape)
        R = np.triu(F)[:k]
        err = np.linalg.norm(R.T @ R - A.T @ A) / np.linalg.norm(A) ** 2
        assert err <= 10 * max(A.shape) * 2.0 ** -53, err
