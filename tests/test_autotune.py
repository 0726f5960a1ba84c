"""The measured autotuner's table on the CPU: size classes, lookup against
the fixed rule, and the save / load round trip (tqr_autotune_run itself, which
times candidates on the device, is covered by a GPU test)."""
import pytest

from paper_0707_3548_gb300 import tqr


@pytest.fixture(autouse=True)
def _clean_table():
    tqr.tqr_autotune_clear()
    yield
    tqr.tqr_autotune_clear()


@pytest.mark.parametrize("m,n,cls", [(1, 1, (0, 0)), (64, 32, (6, 5)), (65, 64, (7, 6)), (128, 100, (7, 7)),
                                     (2048, 2048, (11, 11)), (2049, 1, (12, 0))])
def test_size_classes_are_ceil_log2(m, n, cls):
    assert tqr.tqr_debug_autotune_class(m, n) == cls


def test_untuned_classes_take_the_rule():
    assert tqr.tqr_autotune(2000, 1500) == (128, 16)
    assert tqr.tqr_autotune(100, 40) == (128, 16)
    assert tqr.tqr_autotune(60, 30) == (64, 16)
    assert tqr.tqr_autotune(20, 10) == (32, 16)
    assert tqr.tqr_autotune(9, 9) == (16, 16)


def test_tuned_class_answers_for_every_shape_in_it_and_only_there():
    tqr.tqr_debug_autotune_put(1000, 700, 64, 8)
    assert tqr.tqr_autotune(1000, 700) == (64, 8)
    assert tqr.tqr_autotune(513, 513) == (64, 8)     # same class (10, 10)
    assert tqr.tqr_autotune(1024, 1024) == (64, 8)
    assert tqr.tqr_autotune(1025, 1024) == (128, 16)  # class (11, 10): rule
    assert tqr.tqr_autotune(1000, 400) == (128, 16)   # class (10, 9): rule


def test_save_load_round_trip(tmp_path):
    tqr.tqr_debug_autotune_put(100, 50, 32, 8, 12.5)
    tqr.tqr_debug_autotune_put(2000, 1900, 192, 32, 800.0)
    path = tmp_path / "tune.txt"
    tqr.tqr_autotune_save(str(path))
    text = path.read_text()
    assert "7 6 32 8" in text and "11 11 192 32" in text
    tqr.tqr_autotune_clear()
    assert tqr.tqr_autotune(100, 50) == (128, 16)
    tqr.tqr_autotune_load(str(path))
    assert tqr.tqr_autotune(100, 50) == (32, 8)
    assert tqr.tqr_autotune(2000, 1900) == (192, 32)


def test_malformed_file_is_rejected_whole(tmp_path):
    path = tmp_path / "bad.txt"
    path.write_text("7 6 32 8 1.0\n7 7 48 7 1.0\n")    # ib 7 does not divide 48
    with pytest.raises(tqr.TqrError):
        tqr.tqr_autotune_load(str(path))
    assert tqr.tqr_autotune(100, 50) == (128, 16)       # nothing merged
    with pytest.raises(tqr.TqrError):
        tqr.tqr_autotune_load(str(tmp_path / "missing.txt"))


def test_put_rejects_tiles_the_kernels_cannot_take():
    with pytest.raises(tqr.TqrError):
        tqr.tqr_debug_autotune_put(100, 50, 100, 10)    # nb not a multiple of 8
