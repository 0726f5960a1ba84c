"""The C-ABI library loads and exports every symbol include/*.h declares;
argument validation that happens before any CUDA call."""
import glob
import os
import re

import numpy as np
import pytest

from paper_0707_3548_gb300 import tqr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(tqr_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    return tqr.lib()


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 10
    for name in names:
        assert hasattr(lib, name), name


def test_binding_covers_exactly_the_declarations():
    assert set(tqr.SIGNATURES) == declared_functions()


def test_version(lib):
    assert tqr.tqr_version().startswith("tqr ")


@pytest.mark.parametrize("m,n,nb,ib", [(512, 512, 128, 32), (700, 300, 64, 16), (100, 900, 32, 8), (1, 1, 8, 1)])
def test_t_size_layout(m, n, nb, ib):
    p, q = -(-m // nb), -(-n // nb)
    kt = min(p, q)
    blocks = sum(p - k for k in range(kt))          # (i, k) with k < kt, i >= k
    assert tqr.tqr_t_size(m, n, nb, ib) == blocks * ib * nb * 8


def test_sizes_reject_bad_tiles():
    assert tqr.tqr_t_size(10, 10, 7, 1) == 0        # nb % 8
    assert tqr.tqr_t_size(10, 10, 16, 3) == 0       # ib does not divide nb
    assert tqr.tqr_t_size(10, 10, 512, 64) == 0     # nb > 256
    assert tqr.tqr_t_size(10, 10, 256, 128) == 0    # ib > 64
    assert tqr.tqr_work_size(4096, 4096, 128, 32) > 4096 * 4096 * 8


def test_factor_argument_errors(lib):
    a = np.zeros(16)
    t = np.zeros(16)
    ptr = a.ctypes.data
    assert lib.tqr_factor(-1, 4, ptr, 4, 8, 4, t.ctypes.data, None) == -1
    assert lib.tqr_factor(4, -1, ptr, 4, 8, 4, t.ctypes.data, None) == -2
    assert lib.tqr_factor(4, 4, ptr, 3, 8, 4, t.ctypes.data, None) == -4
    assert lib.tqr_factor(4, 4, ptr, 4, 12, 4, t.ctypes.data, None) == -5
    assert lib.tqr_factor(4, 4, ptr, 4, 16, 5, t.ctypes.data, None) == -6
    assert lib.tqr_factor(4, 4, None, 4, 8, 4, t.ctypes.data, None) == -3
    assert lib.tqr_factor(4, 4, ptr, 4, 8, 4, None, None) == -7
    assert lib.tqr_factor(0, 4, ptr, 1, 8, 4, t.ctypes.data, None) == 0   # empty: nothing to do
    assert lib.tqr_factor_ws(4, 4, ptr, 4, 8, 4, t.ctypes.data, None, 0, None) == -8


def test_apply_and_solve_argument_errors(lib):
    a = np.zeros(16)
    p = a.ctypes.data
    assert lib.tqr_apply_qt(b"X", 4, 4, 1, p, 4, 8, 4, p, p, 4, None) == -1
    assert lib.tqr_apply_qt(b"T", 4, 4, -1, p, 4, 8, 4, p, p, 4, None) == -4
    assert lib.tqr_apply_qt(b"T", 4, 4, 1, p, 4, 8, 4, p, p, 3, None) == -11
    it = tqr.ctypes.c_int(0)
    be = tqr.ctypes.c_double(0)
    args = (p, 4, p, 4, p, 4, 0, 1e-12, 10, tqr.ctypes.byref(it), tqr.ctypes.byref(be), 8, 4, None)
    assert lib.tqr_solve_ls(4, 5, 1, *args) == -2        # n > m
    assert lib.tqr_solve_ls(4, 4, 0, *args) == -3
    bad_prec = (p, 4, p, 4, p, 4, 9, 1e-12, 10, tqr.ctypes.byref(it), tqr.ctypes.byref(be), 8, 4, None)
    assert lib.tqr_solve_ls(4, 4, 1, *bad_prec) == -10
    bad_nb = (p, 4, p, 4, p, 4, 0, 1e-12, 10, tqr.ctypes.byref(it), tqr.ctypes.byref(be), 12, 4, None)
    assert lib.tqr_solve_ls(4, 4, 1, *bad_nb) == -15


def test_debug_schedule_validation(lib):
    assert lib.tqr_debug_set_schedule(3, 0) == -1
    assert lib.tqr_debug_set_schedule(0, -1) == -2
    assert lib.tqr_debug_set_schedule(-1, 0) == 0


def test_debug_shape_override_validation(lib):
    assert lib.tqr_debug_set_shape(12, -1) == -1
    assert lib.tqr_debug_set_shape(0, -2) == -2
    assert lib.tqr_debug_set_shape(16, 4) == 0
    assert lib.tqr_debug_set_shape(0, -1) == 0


def test_debug_trace_rejects_a_negative_capacity():
    import ctypes
    assert tqr.lib().tqr_debug_trace(ctypes.c_void_p(256), -1) == -2


def test_debug_trace_rejects_host_memory():
    import torch
    host = np.zeros((4, 8), dtype=np.int64)
    assert tqr.lib().tqr_debug_trace(host.ctypes.data, 4) == -1
    with pytest.raises(ValueError):
        tqr.tqr_debug_trace(torch.zeros((4, 8), dtype=torch.int64))


def test_trace_decoding_and_chrome_form():
    """Trace words as the kernel writes them (host-built here): decoding keeps
    the written rows, and the Chrome form puts overlapping tasks of one SM on
    separate rows with times from the first ticket."""
    w = np.zeros((4, 8), dtype=np.int64)
    w[0] = [1000, 2000, 5000, 7 | (3 << 16) | (1 << 32), 2, 5, 4, 1 | (6 << 32)]
    w[1] = [1500, 3000, 4000, 7 | (1 << 16), 2, 3, 2, 0]
    w[2] = [1200, 6000, 9000, 8 | (0 << 16), 3, 3, 3, 0]
    r = tqr.trace_records(w)
    assert list(r["sm"]) == [7, 7, 8] and list(r["kind"]) == [3, 1, 0]
    assert list(r["inst"]) == [1, 0, 0] and list(r["s"]) == [1, 0, 0] and list(r["l"]) == [6, 0, 0]
    ev = tqr.trace_chrome(w)["traceEvents"]
    by_name = {e["name"]: e for e in ev}
    assert by_name["SSRFB"]["ts"] == 1.0 and by_name["SSRFB"]["dur"] == 3.0
    assert by_name["SSRFB"]["tid"] != by_name["TSQRT"]["tid"]      # overlap on SM 7
    assert by_name["GEQRT"]["tid"] == 8 * 4 and by_name["GEQRT"]["args"]["wait_us"] == 4.8


def test_trace_summary():
    w = np.zeros((3, 8), dtype=np.int64)
    w[0] = [0, 1000, 5000, 0 | (3 << 16), 0, 1, 1, 0]
    w[1] = [0, 2000, 4000, 1 | (3 << 16), 0, 2, 1, 0]
    w[2] = [500, 5000, 6000, 0 | (0 << 16), 1, 1, 1, 0]
    sm = tqr.trace_summary(w, ctas=2)
    assert sm["tasks"] == 3 and sm["span_us"] == 6.0
    assert sm["kinds"]["SSRFB"] == {"count": 2, "mean_us": 3.0, "total_us": 6.0, "mean_wait_us": 1.5}
    assert sm["kinds"]["GEQRT"]["mean_wait_us"] == 4.5
    assert sm["busy_fraction"] == 7.0 / 12.0
