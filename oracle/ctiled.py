"""ctypes front of oracle/ctiled.c: the paper's multicore tiled QR (the four
tile kernels of Section 3.1 scheduled dynamically over Algorithm 1's DAG,
Section 3.3) on the host's cores.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``): the benchmark's
multithreaded CPU baseline and a second implementation the tests compare with
the NumPy oracle.  ``build()`` compiles the C file with gcc (plain C99 and
POSIX threads, no architecture flags), so it builds the same on x86 and Arm.
"""
import ctypes
import os
import subprocess

import numpy as np

_DIR = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(_DIR, "ctiled.c")
LIB = os.path.join(_DIR, "libctqr.so")
_lib = None


def build(force=False):
    """Compile libctqr.so next to the source if it is missing or stale."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= os.path.getmtime(SRC):
        return LIB
    tmp = LIB + ".tmp"
    cmd = ["gcc", "-O3", "-std=c99", "-fPIC", "-shared", "-pthread", SRC, "-o", tmp, "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("gcc failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
    os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(LIB)
        L.ctqr_factor.restype = ctypes.c_int
        L.ctqr_factor.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                  ctypes.c_int, ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
        _lib = L
    return _lib


def t_blocks(m, n, nb, ib):
    """Number of ib x nb T blocks: one per (i, k), k < min(p, q), i >= k."""
    p, q = -(-m // nb), -(-n // nb)
    return sum(p - k for k in range(min(p, q)))


def tiled_qr(A, nb, ib, threads=None):
    """Factor a copy of A; returns (F, T, seconds): F (m x n) holds R and the
    tiled V as the NumPy oracle's TiledFactors.F[:m, :n], T is the flat array
    of ib x nb blocks (column-major each) in (k, i) order, seconds the wall
    time of the task execution."""
    F = np.array(A, dtype=np.float64, order="F", copy=True)
    m, n = F.shape
    T = np.zeros(t_blocks(m, n, nb, ib) * ib * nb)
    secs = ctypes.c_double(0.0)
    nth = threads or os.cpu_count() or 1
    rc = lib().ctqr_factor(m, n, F.ctypes.data, m, nb, ib, T.ctypes.data, nth, ctypes.byref(secs))
    if rc != 0:
        raise ValueError("ctqr_factor: invalid arguments or out of memory")
    return F, T, secs.value
