"""CPU oracle for the tiled Householder QR of Buttari, Langou, Kurzak and Dongarra.

TEST INFRASTRUCTURE ONLY.  Nothing in the product package may import, call,
link or execute anything under ``oracle/``; only the tests, the smoke check in
``__graft_entry__`` and the ``cpu_baseline`` / ``--impl reference`` legs of
``bench.py`` use it.  The oracle shares no code with the CUDA path.

Everything here is plain NumPy in float64 (float32 only where a function says
so), written for a reader who checks it against the paper by eye:

* ``householder``  -- the reflector, unblocked QR (DGEQR2) and the compact-WY
  ``T`` factor (DLARFT, forward/columnwise), Section 2 of the paper.
* ``tiled``        -- the four tile kernels GEQRT / LARFB / TSQRT / SSRFB
  (Section 3.1) with inner blocking ``ib``, and Algorithm 1 over a zero-padded
  tile grid; applying Q / Q^T from the tiled factors.
* ``dag``          -- the task set of Algorithm 1, its dependency edges
  (Section 3.3) and the per-step operation count (Section 3.2, Eq. opcount).
* ``lstsq``        -- least squares through the QR factors, the normwise
  backward error, and iterative refinement: semi-normal, augmented-system
  (Bjorck) and GMRES-based (Carson, Higham and Pranesh).
* ``ctiled``       -- the paper's multicore design in plain C (ctiled.c): the
  Section 3.1 tile kernels under Section 3.3's dynamic DAG scheduling on
  POSIX threads; the benchmark's multithreaded CPU baseline, checked against
  ``tiled``.

Parity status: every function here is pinned by a ``-m "not gpu"`` test
against something other than itself (closed forms, 50-digit brute force,
LAPACK as a third opinion, invariants); none is "parity unpinned".
"""

from . import householder, tiled, dag, lstsq  # noqa: F401
