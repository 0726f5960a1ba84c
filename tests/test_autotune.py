"""The tile-size autotuner (host only)."""
import pytest

from paper_0707_3548_gb300 import tqr


@pytest.mark.parametrize("m,n", [(1, 1), (64, 32), (300, 150), (2048, 2048), (65536, 2048), (40, 900)])
def test_autotune_returns_supported_tiles(m, n):
    nb, ib = tqr.tqr_autotune(m, n)
    assert 8 <= nb <= 256 and nb % 8 == 0 and 1 <= ib <= 64 and nb % ib == 0
    assert tqr.tqr_t_size(m, n, nb, ib) > 0
    assert tqr.tqr_autotune(m, n) == (nb, ib)   # deterministic


def test_autotune_argument_errors():
    import ctypes
    a = ctypes.c_int(0)
    assert tqr.lib().tqr_autotune(0, 5, ctypes.byref(a), ctypes.byref(a)) == -1
    assert tqr.lib().tqr_autotune(5, 5, None, ctypes.byref(a)) == -3


def test_autotune_rule():
    # measured: nb 128 / ib 16 for every matrix of a batch beat the other choices
    assert tqr.tqr_autotune(2048, 1000) == (128, 16)
    assert tqr.tqr_autotune(129, 40) == (128, 16)
    assert tqr.tqr_autotune(100, 64) == (128, 16)
    assert tqr.tqr_autotune(64, 33) == (64, 16)
    assert tqr.tqr_autotune(10, 3) == (16, 16)
