#!/usr/bin/env python
"""Benchmark of the GB300 tiled Householder QR (libtqr).

Default workload: one 16384 x 16384 FP64 factorization, entries N(0,1) from
NumPy PCG64 seed 0, tile nb = 128, inner block ib = 16 -- the largest square
of the plain-FP64 tiled QR sweep (nb = 128, ib = 16 was the fastest of the
nb in {128, 192, 256} x ib in {16, 32, 64} grid measured at n = 8192) -- with
2b x b bottoms (Section 3.2's non-square blocks: the rows below each diagonal
tile are taken in pairs), the fastest variant at this size.  A step restores
the matrix from a pristine device copy and calls tqr_factor_pairs (pack to
Block Data Layout, the persistent task kernel, unpack).  The 2 GiB input is
larger than L2.  `--workload qr16384` is Algorithm 1's flat b x b tiles.

Metric: TFLOP/s counting 2 m n^2 - 2 n^3 / 3 per factorization, and its
fraction of this GPU's FP64 FMA peak (measured in the run by a DFMA probe).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
    python bench.py --impl reference ...   (the CPU oracle on host cores)

With N > 1 (torchrun) every rank factors its own matrix (independent
replicas, no collective: a single factorization does not shard); value is
the total over ranks divided by the slowest rank's time.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    "qr8192": dict(m=8192, n=8192, nb=128, ib=16),
    "qr16384": dict(m=16384, n=16384, nb=128, ib=16),
    # the small squares take the fastest tiles of the measured sweep (nb in
    # {32 .. 256} x ib in {8 .. 64}): the panel chain, not the updates, bounds them
    "qr4096": dict(m=4096, n=4096, nb=64, ib=8),
    "qr2048": dict(m=2048, n=2048, nb=32, ib=8),
    "ts65536x2048": dict(m=65536, n=2048, nb=128, ib=16),
    # 2b x b bottoms (pairs of tile rows below the diagonal)
    "qr16384_pairs": dict(m=16384, n=16384, nb=128, ib=16, pairs=True),
    "qr8192_pairs": dict(m=8192, n=8192, nb=128, ib=16, pairs=True),
    # the same with the reduction-tree panel (domain size chosen by the library)
    "ts65536x2048_tree": dict(m=65536, n=2048, nb=128, ib=16, tree=True),
    # least squares A = U diag(sigma) V^T, kappa 1e2 / 1e5 / 1e8: plain FP64
    # against FP32 factorization + FP64-residual refinement
    "ls16384x4096k1e2": dict(m=16384, n=4096, nb=128, ib=16, kappa=1e2, ls=True),
    "ls16384x4096k1e5": dict(m=16384, n=4096, nb=128, ib=16, kappa=1e5, ls=True),
    "ls16384x4096k1e8": dict(m=16384, n=4096, nb=128, ib=16, kappa=1e8, ls=True),
    "ls4096x1024k1e2": dict(m=4096, n=1024, nb=128, ib=16, kappa=1e2, ls=True),
    # served least-squares stream: Poisson arrivals, m log-uniform [128, 8192],
    # n uniform [64, m/2], 1-16 right-hand sides, 30% repeat-A, FP64 and
    # refined-FP32 classes, 64 GB HBM budget
    # batched QR: 4096 independent matrices, m log-uniform [64, 2048], n uniform
    # [32, m], N(0,1), tile sizes from the autotuner, one persistent launch
    "batch4096": dict(count=4096, batch=True),
    # Q suite on the 16384 x 16384 factorization: the explicit thin Q
    # (DORGQR analogue) and C Q for a 4096 x 16384 block C (DORMQR analogue,
    # right side)
    # tiled LU with pairwise pivoting (the LU analogue of Algorithm 1)
    "lu16384": dict(m=16384, n=16384, nb=128, ib=16, lu=True),
    "lu8192": dict(m=8192, n=8192, nb=128, ib=16, lu=True),
    "lu16384_pairs": dict(m=16384, n=16384, nb=128, ib=16, lu=True, pairs=True),
    "orgqr16384": dict(m=16384, n=16384, nb=128, ib=16, qsuite="orgqr"),
    "ormqr16384r4096": dict(m=16384, n=16384, nb=128, ib=16, qsuite="ormqr", mc=4096),
    "serve": dict(rate=2000.0, window=1.0, budget=64 << 30, slots=8, pool_bytes=2 << 30, serve=True),
    "serve_low": dict(rate=20.0, window=5.0, budget=64 << 30, slots=8, pool_bytes=2 << 30, serve=True),
}
METRIC = "QR TFLOP/s (2mn^2-2n^3/3) vs FP64 peak"


def qr_flops(m, n):
    k = min(m, n)
    if m >= n:
        return 2.0 * m * n * n - 2.0 * n ** 3 / 3.0
    return 2.0 * n * m * m - 2.0 * m ** 3 / 3.0 if k else 0.0


def workload_name(w):
    extra = ", reduction-tree panel" if w.get("tree") else (", 2b x b bottoms" if w.get("pairs") else "")
    return "tiled QR %dx%d FP64, N(0,1) seed 0, nb=%d ib=%d%s" % (w["m"], w["n"], w["nb"], w["ib"], extra)


# ---------------------------------------------------------------- CPU oracle sample
_ORACLE_SNIPPET = r"""
import json, os, sys, time
sys.path.insert(0, %(root)r)
import numpy as np
from oracle import householder as H
from paper_0707_3548_gb300 import inputs
m, n, target, steps = %(m)d, %(n)d, %(target)f, %(steps)d
FULL = inputs.normal_matrix(m, n, 0)   # the workload matrix (same generator, same seed)
def panel(c):
    return np.asfortranarray(FULL[:, :c])
# calibrate t(c) = a c + b c^2 (per-column overhead + rank-1 updates) at two widths
ts = []
for c in (48, 96):
    t0 = time.perf_counter(); H.geqr2(panel(c)); ts.append(time.perf_counter() - t0)
b = max((ts[1] / 96 - ts[0] / 48) / 48, 1e-12)
a = max(ts[0] / 48 - b * 48, 0.0)
c = (-a + (a * a + 4 * b * target) ** 0.5) / (2 * b)
c = int(max(32, min(n, c)))
P = panel(c)
times = []
for _ in range(steps):
    t0 = time.perf_counter(); H.geqr2(P); times.append(time.perf_counter() - t0)
flops = 2.0 * m * c * c - 2.0 * c ** 3 / 3.0
print(json.dumps({"c": c, "times": times, "flops": flops}))
"""


_CTILED_SNIPPET = r"""
import json, os, platform, subprocess, sys, time
sys.path.insert(0, %(root)r)
import numpy as np
from oracle import ctiled as C
from paper_0707_3548_gb300 import inputs
m, n, nb, ib, target, steps = %(m)d, %(n)d, %(nb)d, %(ib)d, %(target)f, %(steps)d
C.build()
threads = os.cpu_count() or 1
FULL = inputs.normal_matrix(m, n, 0)   # the workload matrix (same generator, same seed)
def flops(c):
    return 2.0 * m * c * c - 2.0 * c ** 3 / 3.0
# calibrate on 4 tile columns, then size c (whole tile columns) for `target`
# seconds assuming time proportional to the flops
c0 = min(n, 4 * nb)
_, _, t0 = C.tiled_qr(np.asfortranarray(FULL[:, :c0]), nb, ib, threads)
rate = flops(c0) / max(t0, 1e-6)
c = c0
while c + nb <= n and flops(c + nb) / rate <= target:
    c += nb
P = np.asfortranarray(FULL[:, :c])
times = []
for _ in range(steps):
    _, _, t = C.tiled_qr(P, nb, ib, threads)
    times.append(t)
model = platform.machine()
try:
    for line in subprocess.run(["lscpu"], capture_output=True, text=True).stdout.splitlines():
        if line.startswith("Model name:"):
            model = line.split(":", 1)[1].strip() + " (" + platform.machine() + ")"
            break
except OSError:
    pass
print(json.dumps({"c": c, "times": times, "flops": flops(c), "threads": threads, "cpu": model}))
"""


def ctiled_sample(m, n, nb, ib, target_s, steps):
    """Times the oracle's multithreaded tiled QR (oracle/ctiled.c: the
    Section 3.1 kernels under Section 3.3's dynamic DAG scheduling, one
    thread per host core) on the first c columns of the workload matrix, c a
    whole number of tile columns sized for ~target_s seconds, in a
    subprocess.  Returns (TFLOP/s per step, c, times, threads, cpu model)."""
    code = _CTILED_SNIPPET % dict(root=ROOT, m=m, n=n, nb=nb, ib=ib, target=target_s, steps=steps)
    env = dict(os.environ)
    env["CUDA_VISIBLE_DEVICES"] = ""
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, check=True)
    r = json.loads(out.stdout.strip().splitlines()[-1])
    rates = [r["flops"] / t / 1e12 for t in r["times"]]
    return rates, r["c"], r["times"], r["threads"], r["cpu"]


def oracle_sample(m, n, target_s, steps):
    """Times the oracle's unblocked Householder QR (DGEQR2 equivalent) on the
    first c columns of the workload matrix, c sized for ~target_s seconds, in
    a single-threaded subprocess.  Returns (TFLOP/s per step, c, times)."""
    code = _ORACLE_SNIPPET % dict(root=ROOT, m=m, n=n, target=target_s, steps=steps)
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[k] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, check=True)
    r = json.loads(out.stdout.strip().splitlines()[-1])
    rates = [r["flops"] / t / 1e12 for t in r["times"]]
    return rates, r["c"], r["times"]


_ORACLE_KIND_SNIPPET = r"""
import json, sys, time
sys.path.insert(0, %(root)r)
import numpy as np
from oracle import householder as H
from oracle import lstsq as LS
from paper_0707_3548_gb300 import inputs
kind, p, target = %(kind)r, json.loads(%(params)r), %(target)f

def fit_cols(make, m, cmax):
    # t(c) = a c + b c^2 from two widths, then c for `target` seconds
    ts = []
    for c in (32, 64):
        X = make(c); t0 = time.perf_counter(); H.geqr2(X); ts.append(time.perf_counter() - t0)
    b = max((ts[1] / 64 - ts[0] / 32) / 32, 1e-12)
    a = max(ts[0] / 32 - b * 32, 0.0)
    return int(max(16, min(cmax, (-a + (a * a + 4 * b * target) ** 0.5) / (2 * b))))

out = {}
if kind == "batch":
    shapes = inputs.batch_shapes(p["count"], seed=0)
    fl, tt, cnt = 0.0, 0.0, 0
    for t, (m, n) in enumerate(shapes):
        A = inputs.normal_matrix(m, n, t)
        t0 = time.perf_counter(); H.geqr2(A); tt += time.perf_counter() - t0
        fl += 2.0 * m * n * n - 2.0 * n ** 3 / 3.0 if m >= n else 2.0 * n * m * m - 2.0 * m ** 3 / 3.0
        cnt += 1
        if tt >= target:
            break
    out = {"flops": fl, "time": tt, "sample": "unblocked Householder QR (oracle) of the first %%d matrices of the batch" %% cnt}
elif kind == "ls":
    m, n, kappa = p["m"], p["n"], p["kappa"]
    c = fit_cols(lambda c: inputs.conditioned_ls_problem(m, c, kappa, seed=0)[0], m, n)
    A, b, _ = inputs.conditioned_ls_problem(m, c, kappa, seed=0)
    t0 = time.perf_counter(); LS.lstsq(A, b[:, None]); tt = time.perf_counter() - t0
    out = {"flops": 2.0 * m * c * c - 2.0 * c ** 3 / 3.0 + 4.0 * m * c, "time": tt,
           "sample": "oracle least squares (unblocked QR, Q^T b, back substitution) of a %%dx%%d problem of the same "
                     "construction (kappa=%%g)" %% (m, c, kappa)}
elif kind == "serve":
    # the stream's requests in arrival order, each solved by the oracle from
    # scratch (no resident factorizations), until the time budget is spent
    reqs, _ = inputs.serving_stream(p["rate"], p["window"], seed=0)
    tt, cnt = 0.0, 0
    for q in reqs:
        A = inputs.normal_matrix(q["m"], q["n"], q["matrix"])
        B = inputs.normal_matrix(q["m"], q["nrhs"], 7 + cnt)
        t0 = time.perf_counter(); LS.lstsq(A, B); tt += time.perf_counter() - t0
        cnt += 1
        if tt >= target:
            break
    out = {"flops": float(cnt), "time": tt,
           "sample": "oracle least squares (unblocked QR) of the stream's first %%d requests in order" %% cnt}
elif kind == "lu":
    from oracle import tiled_lu as TLU
    n = p["n"]
    cs = []
    for c in (96, 192):
        X = inputs.normal_matrix(c, c, 0); t0 = time.perf_counter(); TLU.getrf(X, c); cs.append(time.perf_counter() - t0)
    # t(c) ~ a c^3 (a rank-1 update of the trailing block per column)
    a = max(cs[1] / 192 ** 3, 1e-15)
    c = int(max(32, min(n, (target / a) ** (1.0 / 3.0))))
    X = inputs.normal_matrix(n, n, 0)[:c, :c]
    t0 = time.perf_counter(); TLU.getrf(X, c); tt = time.perf_counter() - t0
    out = {"flops": 2.0 * c ** 3 / 3.0, "time": tt,
           "sample": "oracle partially pivoted LU (GETRF kernel, unblocked) of the leading %%dx%%d block" %% (c, c)}
elif kind in ("orgqr", "ormqr"):
    m = p["m"]
    c = fit_cols(lambda c: inputs.normal_matrix(m, c, 0), m, p["n"])
    F, tau = H.geqr2(inputs.normal_matrix(m, c, 0))
    if kind == "orgqr":
        t0 = time.perf_counter(); H.apply_q(F, tau, np.eye(m, c)); tt = time.perf_counter() - t0
        out = {"flops": 4.0 * m * c * c - 2.0 * (m + c) * c * c + 4.0 * c ** 3 / 3.0, "time": tt,
               "sample": "oracle unblocked Q accumulation of %%d columns from %%d reflectors of length %%d" %% (c, c, m)}
    else:
        r = 64
        C = inputs.normal_matrix(r, m, 1)
        t0 = time.perf_counter(); H.apply_qt(F, tau, C.T); tt = time.perf_counter() - t0
        out = {"flops": 4.0 * r * m * c - 2.0 * r * c * c, "time": tt,
               "sample": "oracle unblocked C Q = (Q^T C^T)^T for %%d rows of C and %%d reflectors of length %%d" %% (r, c, m)}
print(json.dumps(out))
"""


def oracle_kind_sample(kind, params, target_s):
    """Times the oracle on a bounded sample of a non-default workload in a
    single-threaded subprocess; returns (flops, seconds, description)."""
    code = _ORACLE_KIND_SNIPPET % dict(root=ROOT, kind=kind, params=json.dumps(params), target=target_s)
    env = dict(os.environ)
    for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS", "BLIS_NUM_THREADS"):
        env[k] = "1"
    env["CUDA_VISIBLE_DEVICES"] = ""
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, check=True)
    r = json.loads(out.stdout.strip().splitlines()[-1])
    return r["flops"], r["time"], r["sample"]


def run_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    per_step = max(2.0, min(10.0, 120.0 / max(1, args.steps + args.warmup)))
    rates, c, times, threads, cpu_model = ctiled_sample(w["m"], w["n"], w["nb"], w["ib"], per_step,
                                                        args.warmup + args.steps)
    timed = times[args.warmup:]
    rates = rates[args.warmup:]
    value = statistics.mean(rates)
    sample = ("multithreaded tiled QR (oracle/ctiled.c: Section 3.1 kernels, Section 3.3 dynamic DAG "
              "scheduling, %d threads on %s) of the first %d columns of the %dx%d workload matrix per step, "
              "nb=%d ib=%d" % (threads, cpu_model, c, w["m"], w["n"], w["nb"], w["ib"]))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "TFLOP/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * statistics.mean(timed), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic: N(0,1), NumPy PCG64 seed 0",
        "config": {"workload": workload_name(w), "m": w["m"], "n": w["n"], "nb": w["nb"], "ib": w["ib"]},
        "cpu_baseline": {"value": value, "unit": "TFLOP/s", "cores": threads, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- clocks
_SMI_FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
               "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
               "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


class ClockSampler:
    def __init__(self, bus_id):
        self.bus_id = bus_id
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        cmd = ["nvidia-smi", "--query-gpu=" + _SMI_FIELDS, "--format=csv,noheader,nounits", "-lms", "200"]
        if self.bus_id:
            cmd += ["-i", self.bus_id]
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.fh, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not self.path:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 8:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[0]) for r in rows if num(r[0]) is not None]
        mx = [num(r[1]) for r in rows if num(r[1]) is not None]
        pw = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[4 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None, "samples": len(rows), "reasons": reasons}


def engine_sha():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_0707_3548_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.startswith("tqr_engine") or f == "tqr_graph.h":
            with open(os.path.join(csrc, f), "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(workload):
    """DRAM bytes per launch of the task kernel from the committed ncu summary,
    only while the kernel sources still match the capture."""
    path = os.path.join(ROOT, "profiles", "task_kernel_traffic.json")
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path))
    except ValueError:
        return None
    if d.get("engine_sha") != engine_sha():
        return None
    return d.get("traffic_bytes_per_launch", {}).get(workload)


# ---------------------------------------------------------------- main arm
def run_ours(args, w):
    import numpy as np
    import torch

    from paper_0707_3548_gb300 import build as B
    from paper_0707_3548_gb300 import inputs, tqr

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if rank == 0 or world == 1:
        B.build()
    if dist is not None:
        dist.barrier()
    tqr.lib()
    m, n, nb, ib = w["m"], w["n"], w["nb"], w["ib"]
    A = inputs.normal_matrix(m, n, 0)
    dev = torch.device("cuda", local)
    dA0 = tqr.colmajor(torch.from_numpy(A).to(dev))
    dA = tqr.colmajor(torch.empty((m, n), dtype=torch.float64, device=dev))
    tree = bool(w.get("tree"))
    pairs = bool(w.get("pairs"))
    if tree:
        T = torch.zeros(tqr.tqr_t_size_tree(m, n, nb, ib) // 8, dtype=torch.float64, device=dev)
        dA.copy_(dA0)
        _, D = tqr.tqr_factor_tree(dA, nb, ib, 0, T)   # the library's domain choice, reused below
    else:
        T = tqr.new_t(m, n, nb, ib, dA)
        D = 0
    stream = torch.cuda.current_stream()

    def step():
        dA.copy_(dA0)
        if tree:
            tqr.tqr_factor_tree(dA, nb, ib, D, T)
        elif pairs:
            tqr.tqr_factor_pairs(dA, nb, ib, T)
        else:
            tqr.tqr_factor(dA, nb, ib, T)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    assert tqr.tqr_stream_status() == tqr.TQR_OK
    if dist is not None:
        dist.barrier()
    props = torch.cuda.get_device_properties(dev)
    bus = None
    try:
        bus = "%08x:%02x:%02x.0" % (props.pci_domain_id, props.pci_bus_id, props.pci_device_id)
    except AttributeError:
        bus = None
    tqr.tqr_debug_timing(1)
    tqr.tqr_debug_timing_read()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(bus) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
    kern_ms, launches = tqr.tqr_debug_timing_read()
    tqr.tqr_debug_timing(0)
    status = tqr.tqr_stream_status()
    elapsed_ms = e0.elapsed_time(e1)
    from paper_0707_3548_gb300.ranks import max_over_ranks
    elapsed_ms = max_over_ranks(elapsed_ms, dist, dev)
    flops = qr_flops(m, n)
    value = flops * args.steps * world / (elapsed_ms * 1e-3) / 1e12

    # end to end through the C ABI with pinned host buffers
    hA_t = torch.empty((n, m), dtype=torch.float64).pin_memory()
    hA = hA_t.numpy().T                       # column-major m x n view
    hT_t = torch.empty(T.numel(), dtype=torch.float64).pin_memory()
    hT = hT_t.numpy()
    e2e_times = []
    for it in range(0 if args.no_e2e else args.warmup + args.steps):
        np.copyto(hA, A)
        t0 = time.perf_counter()
        if tree:
            tqr.tqr_factor_tree(hA, nb, ib, D, hT)
        elif pairs:
            tqr.tqr_factor_pairs(hA, nb, ib, hT)
        else:
            tqr.tqr_factor(hA, nb, ib, hT)
        t1 = time.perf_counter()
        if it >= args.warmup:
            e2e_times.append(t1 - t0)
    e2e_s = statistics.mean(e2e_times) if e2e_times else float("nan")
    if e2e_times:
        e2e_s = max_over_ranks(e2e_s, dist, dev)
    e2e = None
    if e2e_times:
        e2e = {"value": flops * world / e2e_s / 1e12, "unit": "TFLOP/s",
               "h2d_bytes_per_step": 8 * m * n, "d2h_bytes_per_step": 8 * m * n + 8 * T.numel(),
               "ms_per_step": e2e_s * 1e3}

    peak = tqr.tqr_debug_fp64_peak()
    kern_avg_ms = kern_ms / max(1, launches)
    achieved = flops / (kern_avg_ms * 1e-3) / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": measured_traffic(args.workload),
                "kernel": ("tqr::run_pair_tasks_kernel<double>" if pairs else "tqr::run_tasks_kernel<double>") +
                          " (persistent task scheduler)",
                "peak_source": "FP64 DFMA probe measured in this run (tqr_debug_fp64_peak); "
                               "nominal GB300 FP64 1.25 TFLOP/s",
                "kernel_ms_per_launch": kern_avg_ms}

    if rank != 0:
        if dist is not None:
            dist.barrier()
            dist.destroy_process_group()
        return
    # the least-squares half of the metric: plain FP64 against FP32 +
    # refinement on the 16384 x 4096, kappa = 1e2 problem, equal error 1e-12
    ls = None
    if world == 1 and not args.no_ls:
        dA = dA0 = T = None
        torch.cuda.empty_cache()
        ls = ls_measure(16384, 4096, 1e2, 128, 16, 1, 2)
        ls["workload"] = "least squares 16384x4096, A = U diag(sigma) V^T, kappa 1e2, nrhs 1, nb 128 ib 16, seed 0"
    cpu = cpu1 = None
    if world == 1 and not args.no_cpu_baseline:
        rates, c, times, threads, cpu_model = ctiled_sample(m, n, nb, ib, 12.0, 2)
        cpu = {"value": max(rates), "unit": "TFLOP/s", "cores": threads, "kind": "oracle",
               "sample": "multithreaded tiled QR (oracle/ctiled.c: Section 3.1 kernels, Section 3.3 dynamic DAG "
                         "scheduling, %d threads on %s) of the first %d columns of the %dx%d workload matrix, "
                         "nb=%d ib=%d, best of 2 (%.1f s)" % (threads, cpu_model, c, m, n, nb, ib, min(times))}
        rates, c, times = oracle_sample(m, n, 4.0, 1)
        cpu1 = {"value": max(rates), "unit": "TFLOP/s", "cores": 1, "kind": "oracle",
                "sample": "unblocked Householder QR (oracle, NumPy fp64, 1 thread) of the first %d columns of the "
                          "%dx%d workload matrix (%.1f s)" % (c, m, n, min(times))}
    line = {
        "metric": METRIC, "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic: N(0,1) entries, NumPy PCG64 seed 0",
        "config": {"workload": workload_name(w), "m": m, "n": n, "nb": nb, "ib": ib,
                   "l2": "input 8*m*n bytes > 129 MB L2, restored from a device copy each step",
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "panel": ("reduction tree, domains of %d tile rows" % D) if tree else
                            ("flat, 2b x b bottoms (pairs of tile rows)" if pairs else "flat (Algorithm 1)")},
        "fp64_peak_fraction": value / world / peak,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "cpu_baseline_unblocked_1thread": cpu1,
        "e2e": e2e,
        "gpu_launches": 3 * args.steps,
        "clocks": clk.summary(),
        "status": status,
        "ls": ls,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def ls_measure(m, n, kappa, nb, ib, warmup, steps, problem=None):
    """One least-squares problem (A = U diag(sigma) V^T, seed 0, one right-hand
    side) solved by tqr_solve_ls in plain FP64 and in FP32 + refinement, both
    to backward error 1e-12: wall time per solve (device buffers, stream
    synchronized), the device-reported and the host-recomputed backward
    errors, and the refinement path."""
    import numpy as np
    import torch

    from paper_0707_3548_gb300 import inputs, tqr

    A, b, _ = problem if problem is not None else inputs.conditioned_ls_problem(m, n, kappa, seed=0)
    dA = tqr.colmajor(torch.from_numpy(A).cuda())
    db = tqr.colmajor(torch.from_numpy(b[:, None]).cuda())
    out = {}
    xs = {}
    for name, prec in (("fp64", tqr.TQR_PREC_FP64), ("fp32_refined", tqr.TQR_PREC_FP32)):
        times, its, berrs, rcs = [], [], [], []
        info = {}
        for step in range(warmup + steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            X, it, berr, rc = tqr.tqr_solve_ls(dA, db, prec=prec, tol=1e-12, maxit=40, nb=nb, ib=ib, check=False)
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            info = tqr.tqr_ls_last_info()
            if step >= warmup:
                times.append(t1 - t0)
                its.append(it)
                berrs.append(berr)
                rcs.append(rc)
        xs[name] = X.cpu().numpy()[:, 0]
        r = b - A @ xs[name]
        nA = float(np.linalg.norm(A))
        host_berr = float(np.linalg.norm(A.T @ r) / (nA * (nA * np.linalg.norm(xs[name]) + np.linalg.norm(b))))
        lat = sorted(times)
        out[name] = {"ms": 1e3 * statistics.mean(times), "solves_per_s": 1.0 / statistics.mean(times),
                     "p50_ms": 1e3 * lat[len(lat) // 2],
                     "p99_ms": 1e3 * lat[min(len(lat) - 1, int(0.99 * len(lat)))], "iters": its[-1],
                     "inner_iters": info.get("inner_iters"), "path": info.get("path"),
                     "berr": max(berrs), "berr_host": host_berr, "status": rcs[-1]}
    ref = xs["fp64"]
    out["fp32_refined"]["rel_diff_vs_fp64"] = float(np.linalg.norm(xs["fp32_refined"] - ref) / np.linalg.norm(ref))
    out["speedup_vs_fp64"] = out["fp64"]["ms"] / out["fp32_refined"]["ms"]
    out["equal_error"] = bool(out["fp64"]["berr_host"] <= 1e-12 and out["fp32_refined"]["berr_host"] <= 1e-12)
    return out


def run_ls(args, w):
    """Least-squares solves/s, plain FP64 vs FP32 + refinement, same problem,
    same backward-error target (1e-12)."""
    import torch

    from paper_0707_3548_gb300 import build as B

    torch.cuda.set_device(0)
    B.build()
    m, n, nb, ib = w["m"], w["n"], w["nb"], w["ib"]
    out = ls_measure(m, n, w["kappa"], nb, ib, args.warmup, args.steps)
    cpu = None
    if not args.no_cpu_baseline:
        fl, tt, smp = oracle_kind_sample("ls", {"m": m, "n": n, "kappa": w["kappa"]}, 8.0)
        full = 2.0 * m * n * n - 2.0 * n ** 3 / 3.0 + 4.0 * m * n
        cpu = {"value": fl / tt / full, "unit": "solves/s", "cores": 1, "kind": "oracle",
               "sample": smp + ", %.1f s; scaled to this workload by its flop count" % tt}
    line = {"metric": "LS solves/s, plain FP64 vs FP32+refinement at backward error <= 1e-12",
            "value": out["fp32_refined"]["solves_per_s"], "unit": "solves/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic: A = U diag(sigma) V^T, seed 0",
            "config": {"workload": "least squares %dx%d kappa=%g, nrhs=1, nb=%d ib=%d" % (m, n, w["kappa"], nb, ib)},
            "ls": out, "speedup_vs_fp64": out["speedup_vs_fp64"],
            "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)


def run_qsuite(args, w):
    """tqr_orgqr (explicit thin Q) or tqr_ormqr (C Q, right side) on a
    factorization made once before the timed region.  LAPACK's operation
    counts: DORGQR 4 m c k - 2 (m + c) k^2 + 4 k^3 / 3 (c columns, k
    reflector columns), DORMQR right side 4 mc m k - 2 mc k^2."""
    import numpy as np
    import torch

    from paper_0707_3548_gb300 import build as B
    from paper_0707_3548_gb300 import inputs, tqr

    torch.cuda.set_device(0)
    B.build()
    m, n, nb, ib = w["m"], w["n"], w["nb"], w["ib"]
    k = min(m, n)
    A = inputs.normal_matrix(m, n, 0)
    dA = tqr.colmajor(torch.from_numpy(A).cuda())
    T = tqr.tqr_factor(dA, nb, ib)
    org = w["qsuite"] == "orgqr"
    if org:
        c = n
        out = tqr.colmajor(torch.empty((m, c), dtype=torch.float64, device="cuda"))
        flops = 4.0 * m * c * k - 2.0 * (m + c) * k * k + 4.0 * k ** 3 / 3.0
        name = "explicit thin Q (%dx%d) of the tiled QR of a %dx%d N(0,1) matrix, nb=%d ib=%d" % (m, c, m, n, nb, ib)
        metric = "DORGQR-analogue TFLOP/s (4mck-2(m+c)k^2+4k^3/3) vs FP64 peak"

        def step():
            tqr.tqr_orgqr(dA, nb, ib, T, c, Q=out)
    else:
        mc = w["mc"]
        C0 = tqr.colmajor(torch.from_numpy(inputs.normal_matrix(mc, m, 1)).cuda())
        out = torch.empty_like(C0)
        out = tqr.colmajor(out)
        flops = 4.0 * mc * m * k - 2.0 * mc * k * k
        name = "C Q, C %dx%d N(0,1), Q of the tiled QR of a %dx%d N(0,1) matrix, nb=%d ib=%d" % (mc, m, m, n, nb, ib)
        metric = "DORMQR-analogue TFLOP/s (right side, 4 mc m k - 2 mc k^2) vs FP64 peak"

        def step():
            out.copy_(C0)
            tqr.tqr_ormqr("R", "N", dA, nb, ib, T, out)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    assert tqr.tqr_stream_status() == tqr.TQR_OK
    props = torch.cuda.get_device_properties(0)
    try:
        bus = "%08x:%02x:%02x.0" % (props.pci_domain_id, props.pci_bus_id, props.pci_device_id)
    except AttributeError:
        bus = None
    tqr.tqr_debug_timing(1)
    tqr.tqr_debug_timing_read()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(bus) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
    kern_ms, launches = tqr.tqr_debug_timing_read()
    tqr.tqr_debug_timing(0)
    status = tqr.tqr_stream_status()
    elapsed_ms = e0.elapsed_time(e1)
    value = flops * args.steps / (elapsed_ms * 1e-3) / 1e12
    # end to end with host buffers (A, T and the operand copied in, the result out)
    e2e = None
    if not args.no_e2e:
        hA, hT = dA.cpu().numpy(), T.cpu().numpy()
        hA = np.asfortranarray(hA)
        hO = np.asfortranarray(out.cpu().numpy())
        hC0 = None if org else np.asfortranarray(C0.cpu().numpy())
        ts = []
        for it in range(args.warmup + args.steps):
            if not org:
                np.copyto(hO, hC0)
            t0 = time.perf_counter()
            if org:
                tqr.tqr_orgqr(hA, nb, ib, hT, n, Q=hO)
            else:
                tqr.tqr_ormqr("R", "N", hA, nb, ib, hT, hO)
            if it >= args.warmup:
                ts.append(time.perf_counter() - t0)
        sec = statistics.mean(ts)
        h2d = 8 * (m * n + hT.size) + (0 if org else 8 * hO.size)
        e2e = {"value": flops / sec / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": 8 * hO.size, "ms_per_step": 1e3 * sec}
    cpu = None
    if not args.no_cpu_baseline:
        fl, tt, smp = oracle_kind_sample(w["qsuite"], {"m": m, "n": n}, 8.0)
        cpu = {"value": fl / tt / 1e12, "unit": "TFLOP/s", "cores": 1, "kind": "oracle",
               "sample": smp + ", %.1f s" % tt}
    peak = tqr.tqr_debug_fp64_peak()
    kern_avg_ms = kern_ms / max(1, launches)
    achieved = flops / (kern_avg_ms * 1e-3) / 1e12
    line = {"metric": metric, "value": value, "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic: N(0,1), NumPy PCG64",
            "config": {"workload": name, "m": m, "n": n, "nb": nb, "ib": ib, "flops_per_step": flops,
                       "l2": "operands (2 GiB A, %d MiB result) > 129 MB L2" % (8 * out.numel() >> 20)},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": measured_traffic(args.workload),
                         "kernel": "tqr::run_tasks_kernel<double> (persistent task scheduler)",
                         "peak_source": "FP64 DFMA probe measured in this run (tqr_debug_fp64_peak)",
                         "kernel_ms_per_launch": kern_avg_ms},
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": 4 * args.steps,
            "clocks": clk.summary(), "status": status}
    print(json.dumps(line), flush=True)


def run_lu(args, w):
    """Tiled LU (pairwise pivoting): value = 2n^3/3 per factorization (LAPACK's
    count for n x n) over the timed steps; each step restores A from a device
    copy and calls tqr_lu_factor."""
    import torch

    from paper_0707_3548_gb300 import build as B
    from paper_0707_3548_gb300 import inputs, tqr

    torch.cuda.set_device(0)
    B.build()
    m, n, nb, ib = w["m"], w["n"], w["nb"], w["ib"]
    A = inputs.normal_matrix(m, n, 0)
    dA0 = tqr.colmajor(torch.from_numpy(A).cuda())
    dA = tqr.colmajor(torch.empty_like(dA0))
    L = tqr.new_t(m, n, nb, ib, dA)
    piv = torch.zeros(tqr.tqr_lu_piv_size(m, n, nb) // 4, dtype=torch.int32, device="cuda")
    k = min(m, n)
    flops = 2.0 * k ** 3 / 3.0 + (m - k) * k * k + (n - k) * k * k   # LAPACK DGETRF (equals 2n^3/3 if square)
    stream = torch.cuda.current_stream()

    pairs = bool(w.get("pairs"))

    def step():
        dA.copy_(dA0)
        tqr.tqr_lu_factor(dA, nb, ib, L, piv, pairs=pairs)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    props = torch.cuda.get_device_properties(0)
    try:
        bus = "%08x:%02x:%02x.0" % (props.pci_domain_id, props.pci_bus_id, props.pci_device_id)
    except AttributeError:
        bus = None
    tqr.tqr_debug_timing(1)
    tqr.tqr_debug_timing_read()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(bus) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            step()
        e1.record(stream)
        torch.cuda.synchronize()
    kern_ms, launches = tqr.tqr_debug_timing_read()
    tqr.tqr_debug_timing(0)
    status = tqr.tqr_stream_status()
    elapsed_ms = e0.elapsed_time(e1)
    value = flops * args.steps / (elapsed_ms * 1e-3) / 1e12
    e2e = None
    if not args.no_e2e:
        import numpy as np
        hA = np.asfortranarray(A)
        hL = L.cpu().numpy()
        hp = piv.cpu().numpy()
        ts = []
        for it in range(args.warmup + args.steps):
            np.copyto(hA, A)
            t0 = time.perf_counter()
            tqr.tqr_lu_factor(hA, nb, ib, hL, hp, pairs=pairs)
            if it >= args.warmup:
                ts.append(time.perf_counter() - t0)
        sec = statistics.mean(ts)
        e2e = {"value": flops / sec / 1e12, "unit": "TFLOP/s", "h2d_bytes_per_step": 8 * m * n,
               "d2h_bytes_per_step": 8 * m * n + 8 * hL.size + 4 * hp.size, "ms_per_step": 1e3 * sec}
    cpu = None
    if not args.no_cpu_baseline:
        fl, tt, smp = oracle_kind_sample("lu", {"n": n}, 8.0)
        cpu = {"value": fl / tt / 1e12, "unit": "TFLOP/s", "cores": 1, "kind": "oracle",
               "sample": smp + ", %.1f s" % tt}
    peak = tqr.tqr_debug_fp64_peak()
    kern_avg_ms = kern_ms / max(1, launches)
    achieved = flops / (kern_avg_ms * 1e-3) / 1e12
    line = {"metric": "LU TFLOP/s (2n^3/3) vs FP64 peak", "value": value, "unit": "TFLOP/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic: N(0,1) entries, NumPy PCG64 seed 0",
            "config": {"workload": "tiled LU (pairwise pivoting) %dx%d FP64, N(0,1) seed 0, nb=%d ib=%d%s"
                                   % (m, n, nb, ib, ", 2b x b bottoms" if pairs else ""),
                       "m": m, "n": n, "nb": nb, "ib": ib,
                       "l2": "input 8*m*n bytes > 129 MB L2, restored from a device copy each step"},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": measured_traffic(args.workload),
                         "kernel": "tqr::run_lu_tasks_kernel<double> (persistent task scheduler)",
                         "peak_source": "FP64 DFMA probe measured in this run (tqr_debug_fp64_peak)",
                         "kernel_ms_per_launch": kern_avg_ms},
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": 3 * args.steps, "clocks": clk.summary(),
            "status": status}
    print(json.dumps(line), flush=True)


def run_batch(args, w):
    """Batched factorization: all matrices of a rank in one persistent launch
    (CUDA graph), value = total 2mn^2 - 2n^3/3 over the batch / device time.
    With N ranks the matrices are sharded by flops (greedy, no collective);
    the job's time is the slowest rank's."""
    import numpy as np
    import torch

    from paper_0707_3548_gb300 import build as B
    from paper_0707_3548_gb300 import inputs, tqr
    from paper_0707_3548_gb300.ranks import max_over_ranks, shard_by_cost

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if rank == 0 or world == 1:
        B.build()
    if dist is not None:
        dist.barrier()
    all_shapes = inputs.batch_shapes(w["count"], seed=0)
    all_flops = [qr_flops(m, n) for m, n in all_shapes]
    mine = shard_by_cost(all_flops, world)[rank]
    shapes = [all_shapes[t] for t in mine]
    flops = sum(all_flops)
    pristine = []
    for t in mine:
        m, n = all_shapes[t]
        A = inputs.normal_matrix(m, n, t)
        pristine.append(tqr.colmajor(torch.from_numpy(A).to(dev)))
    work = [tqr.colmajor(torch.empty_like(a)) for a in pristine]
    tune_s = 0.0
    rule_tiles = None
    tqr.tqr_autotune_clear()
    if "nb" in w:   # --nb/--ib: one tile shape for every matrix instead of the autotuner's
        tiles = [(min(w["nb"], max(16, 1 << (max(m, n) - 1).bit_length())), w["ib"]) for m, n in shapes]
        tiles = [(nb, min(ib, nb)) for nb, ib in tiles]
    else:
        rule_tiles = [tqr.tqr_autotune(m, n) for m, n in shapes]
        # the measured autotuner: every size class present in this rank's share
        t0 = time.perf_counter()
        if args.tune_cache and os.path.exists(args.tune_cache):
            tqr.tqr_autotune_load(args.tune_cache)
        # per-class measurements, then the tile policy measured on this batch
        tqr.tqr_autotune_batch(shapes)
        if args.tune_cache:
            tqr.tqr_autotune_save(args.tune_cache)
        tune_s = time.perf_counter() - t0
        tiles = [tqr.tqr_autotune(m, n) for m, n in shapes]
    stream = torch.cuda.current_stream()
    props = torch.cuda.get_device_properties(dev)
    try:
        bus = "%08x:%02x:%02x.0" % (props.pci_domain_id, props.pci_bus_id, props.pci_device_id)
    except AttributeError:
        bus = None

    def restore():
        for a, b in zip(work, pristine):
            a.copy_(b)

    # 2b x b bottoms by default (as the single-matrix headline); --variant flat
    # gives Algorithm 1's b x b tiles
    pairs = args.variant != "flat"

    def timed(tl, clk_sampler, pairs=pairs):
        Ts = [torch.zeros(tqr.tqr_t_size(m, n, nb, ib) // 8, dtype=torch.float64, device=dev)
              for (m, n), (nb, ib) in zip(shapes, tl)]
        t_plan = time.perf_counter()
        restore()
        rc, st = tqr.tqr_batch_wait(tqr.tqr_batch_submit(work, Ts, tl, pairs=pairs), len(shapes))
        t_plan = time.perf_counter() - t_plan
        assert rc == 0
        for _ in range(args.warmup - 1):
            restore()
            tqr.tqr_batch_wait(tqr.tqr_batch_submit(work, Ts, tl, pairs=pairs), len(shapes))
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        total = 0.0
        with clk_sampler as clk:
            for _ in range(args.steps):
                restore()
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                t = tqr.tqr_batch_submit(work, Ts, tl, pairs=pairs)
                e1.record(stream)
                rc, st = tqr.tqr_batch_wait(t, len(shapes))
                torch.cuda.synchronize()
                assert rc == 0 and not st.any()
                total += e0.elapsed_time(e1) * 1e-3
        if dist is not None:
            dist.barrier()
        return max_over_ranks(total / args.steps, dist, dev), t_plan, clk

    rule_sec = None
    if rule_tiles is not None and rule_tiles != tiles:
        rule_sec, _, _ = timed(rule_tiles, ClockSampler(None))
    bxb_sec = timed(tiles, ClockSampler(None), pairs=False)[0] if pairs else None
    sec, t_plan, clk = timed(tiles, ClockSampler(bus))
    if rank != 0:
        dist.destroy_process_group()
        return
    classes = {}
    for nb, ib in tiles:
        classes["%d/%d" % (nb, ib)] = classes.get("%d/%d" % (nb, ib), 0) + 1
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        fl, tt, smp = oracle_kind_sample("batch", {"count": w["count"]}, 8.0)
        cpu = {"value": fl / tt / 1e12, "unit": "TFLOP/s", "cores": 1, "kind": "oracle",
               "sample": smp + ", %.1f s" % tt}
    line = {"metric": METRIC + " (batched)", "value": flops / sec / 1e12, "unit": "TFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sec, "higher_is_better": True,
            "scaling": "strong" if world > 1 else "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic: N(0,1), seed per matrix",
            "config": {"workload": "batched QR of %d matrices, m log-uniform [64, 2048], n uniform [32, m], one "
                                   "persistent launch per rank, autotuned nb/ib" % len(all_shapes),
                       "total_flops": flops, "total_bytes": 8 * sum(m * n for m, n in all_shapes),
                       "l2": "inputs > 129 MB L2, restored from device copies before each step",
                       "parallelism": ("instances sharded over %d ranks by flops (greedy), no collective" % world)
                                      if world > 1 else "single GPU",
                       "tile_classes_rank0": classes,
                       "variant": "2b x b bottoms (tqr_batch_submit_pairs)" if pairs else "b x b tiles",
                       "autotune": "measured per size class and per batch policy (tqr_autotune_batch), %.1f s"
                                   % tune_s
                                   if rule_tiles is not None else "fixed by --nb/--ib"},
            "rule_tiles_value": flops / rule_sec / 1e12 if rule_sec else None,
            "bxb_tiles_value": flops / bxb_sec / 1e12 if bxb_sec else None,
            "first_submit_s_incl_plan": t_plan, "gpu_launches": 3 * args.steps, "cpu_baseline": cpu,
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_serve(args, w):
    """Open-loop request stream against the LS server.  The timed region runs
    from the first submission to the last completion; latency is submit to
    completion per request (server clock)."""
    import threading

    import numpy as np
    import torch

    from paper_0707_3548_gb300 import build as B
    from paper_0707_3548_gb300 import inputs, tqr

    from paper_0707_3548_gb300.ranks import max_over_ranks, route_requests

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    if rank == 0 or world == 1:
        B.build()
    if dist is not None:
        dist.barrier()
    rate = args.rate or w["rate"]
    window = args.window or w["window"]
    all_reqs, mats = inputs.serving_stream(rate, window, seed=0)
    if args.classes != "mixed":    # the whole stream in one precision class
        for q in all_reqs:
            q["prec"] = args.classes
    # requests are routed to ranks by matrix affinity / least load (every
    # rank computes the same routing; no data moves between ranks)
    route, _ = route_requests(all_reqs, world)
    reqs = [q for q, r in zip(all_reqs, route) if r == rank]
    mine_ids = {q["matrix"] for q in reqs}
    mats = [x for x in mats if x[2] in mine_ids]
    # distinct matrix data is drawn into a bounded pool; a later matrix id
    # reuses the leading m x n block of the smallest pool matrix that covers
    # it (its own identity is kept: a new id is factored again)
    pool, view_of, used = [], {}, 0
    for m, n, mid in mats:
        cover = [k for k, d in enumerate(pool) if d.shape[0] >= m and d.shape[1] >= n]
        if used + 8 * m * n > w["pool_bytes"] and cover:
            k = min(cover, key=lambda k: pool[k].numel())
            view_of[mid] = pool[k][:m, :n]
            continue
        A = inputs.normal_matrix(m, n, 10_000 + mid)
        pool.append(tqr.colmajor(torch.from_numpy(A).to(dev)))
        used += 8 * m * n
        view_of[mid] = pool[-1]
    rhs = []
    for r, q in enumerate(reqs):
        Bh = inputs.normal_matrix(q["m"], q["nrhs"], 50_000 + r)
        rhs.append(tqr.colmajor(torch.from_numpy(Bh).to(dev)))
    outs = [tqr.colmajor(torch.zeros((q["n"], q["nrhs"]), dtype=torch.float64, device=dev)) for q in reqs]
    torch.cuda.synchronize()
    srv = tqr.Server(w["budget"], slots=w["slots"], grid_cap=args.grid_cap)
    # warm the plan cache and kernels with a few requests outside the window
    for k, q in enumerate(reqs[:3]):
        Xw = tqr.colmajor(torch.zeros((q["n"], q["nrhs"]), dtype=torch.float64, device=dev))
        srv.wait(srv.submit(10**9 + q["matrix"], view_of[q["matrix"]], rhs[k], Xw,
                            prec=tqr.TQR_PREC_FP32 if q["prec"] == "fp32r" else tqr.TQR_PREC_FP64))
    base = srv.stats()
    ids = [None] * len(reqs)
    if dist is not None:
        dist.barrier()
    t0 = time.perf_counter()

    def feeder():
        for k, q in enumerate(reqs):
            dt = q["t"] - (time.perf_counter() - t0)
            if dt > 0:
                time.sleep(dt)
            ids[k] = srv.submit(q["matrix"], view_of[q["matrix"]], rhs[k], outs[k],
                                prec=tqr.TQR_PREC_FP32 if q["prec"] == "fp32r" else tqr.TQR_PREC_FP64)

    th = threading.Thread(target=feeder)
    th.start()
    th.join()
    infos = [srv.wait(r) for r in ids]
    t1 = time.perf_counter()
    last_failure = srv.last_failure()
    span = max_over_ranks(t1 - t0, dist, dev)
    if dist is not None:
        # per-request records (latency, status, class, backward error) to rank 0
        recs = [(i["latency_ms"], i["status"], q["prec"], i["berr"], i["iters"], q["m"], q["n"], i.get("reused", 0))
                for i, q in zip(infos, reqs)]
        gathered = [None] * world
        dist.all_gather_object(gathered, recs)
        stats = srv.stats()
        srv.close()
        if rank != 0:
            dist.destroy_process_group()
            return
        recs = [x for g in gathered for x in g]
        infos = [dict(latency_ms=x[0], status=x[1], berr=x[3], iters=x[4], reused=x[7]) for x in recs]
        reqs = [dict(prec=x[2], m=x[5], n=x[6]) for x in recs]
        t1 = t0 + span
    failures = {}
    for i, q in zip(infos, reqs):
        if i["status"] != 0:
            key = "%s status %d" % (q["prec"], i["status"])
            failures[key] = failures.get(key, 0) + 1
    if dist is None:
        stats = srv.stats()
        srv.close()
    lat = {c: sorted(i["latency_ms"] for i, q in zip(infos, reqs) if q["prec"] == c) for c in ("fp64", "fp32r")}
    def pct(v, p):
        return v[min(len(v) - 1, int(p * (len(v) - 1) + 0.5))] if v else None
    allv = sorted(i["latency_ms"] for i in infos)
    bad = sum(1 for i in infos if i["status"] != 0)
    # what the slowest requests are: their sizes against the stream's (a tail
    # of the largest factorizations is service time, one of small requests
    # would be queueing)
    work = sorted(2.0 * q["m"] * q["n"] ** 2 for q in reqs)
    def work_rank(q):
        import bisect
        return bisect.bisect_left(work, 2.0 * q["m"] * q["n"] ** 2) / max(1, len(work) - 1)
    thr = pct(allv, 0.99)
    tail = [(i, q) for i, q in zip(infos, reqs) if thr is not None and i["latency_ms"] >= thr]
    tail_info = None
    if tail:
        ranks = sorted(work_rank(q) for _, q in tail)
        tail_info = {"requests": len(tail), "median_m": sorted(q["m"] for _, q in tail)[len(tail) // 2],
                     "median_n": sorted(q["n"] for _, q in tail)[len(tail) // 2],
                     "fresh_fraction": sum(1 for i, _ in tail if not i.get("reused")) / len(tail),
                     "median_work_percentile": ranks[len(ranks) // 2]}
    buckets = {}
    for lo, hi in ((128, 512), (512, 2048), (2048, 8193)):
        v = sorted(i["latency_ms"] for i, q in zip(infos, reqs) if lo <= q["m"] < hi)
        buckets["m %d-%d" % (lo, hi - 1)] = {"count": len(v), "p50_ms": pct(v, 0.5), "p99_ms": pct(v, 0.99)}
    line = {"metric": "LS solves/s + p99 latency (served stream)", "value": len(reqs) / (t1 - t0), "unit": "solves/s",
            "n_gpus": world, "steps": 1, "warmup": 3, "ms_per_step": 1e3 * (t1 - t0), "higher_is_better": True,
            "scaling": "strong" if world > 1 else "weak", "vs_baseline": None,
            "dtype": {"mixed": "f64 / f32+f64 refined", "fp64": "f64", "fp32r": "f32+f64 refined"}[args.classes],
            "data": "synthetic: Poisson stream seed 0; matrix data from a %.1f GB pool" % (w["pool_bytes"] / 2**30),
            "config": {"workload": "served LS stream %.0f req/s for %.1f s, %d requests, budget %d GB, %d slots, "
                                   "classes %s" % (rate, window, len(reqs), w["budget"] >> 30, w["slots"], args.classes),
                       "parallelism": ("requests routed over %d ranks (matrix affinity, least load), no data "
                                       "collective" % world) if world > 1 else "single GPU"},
            "offered_per_s": len(reqs) / window, "completed": len(reqs) - bad, "failed": bad,
            "failures": failures, "last_failure": last_failure or None, "slots": w["slots"],
            "grid_cap": args.grid_cap,
            "p50_ms": pct(allv, 0.5), "p99_ms": pct(allv, 0.99),
            "classes": {c: {"count": len(v), "p50_ms": pct(v, 0.5), "p99_ms": pct(v, 0.99)} for c, v in lat.items()},
            "reused_resident": stats["reused"] - base["reused"],
            "max_iters_fp32r": max([i["iters"] for i, q in zip(infos, reqs) if q["prec"] == "fp32r"] or [0]),
            "max_berr": max(i["berr"] for i in infos),
            "p99_tail": tail_info, "latency_by_m": buckets}
    if not args.no_cpu_baseline and world == 1:
        cnt, tt, smp = oracle_kind_sample("serve", {"rate": rate, "window": window}, 8.0)
        line["cpu_baseline"] = {"value": cnt / tt, "unit": "solves/s", "cores": 1, "kind": "oracle",
                                "sample": smp + ", %.1f s" % tt}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="qr16384_pairs", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end measurement")
    ap.add_argument("--no-ls", action="store_true", help="skip the least-squares comparison of the default line")
    ap.add_argument("--classes", default="mixed", choices=["mixed", "fp64", "fp32r"],
                    help="serve: precision classes of the stream (mixed 50/50, or all one class)")
    ap.add_argument("--tune-cache", default="", help="batch: autotuner table file to load before and save after")
    ap.add_argument("--variant", default="", choices=["", "flat", "pairs", "tree"],
                    help="override the factorization variant of a QR workload")
    ap.add_argument("--nb", type=int, default=0, help="override the workload's tile size")
    ap.add_argument("--ib", type=int, default=0, help="override the workload's inner block size")
    ap.add_argument("--rate", type=float, default=0.0, help="serve: arrival rate (req/s)")
    ap.add_argument("--window", type=float, default=0.0, help="serve: arrival window (s)")
    ap.add_argument("--slots", type=int, default=0, help="serve: concurrent request slots")
    ap.add_argument("--grid-cap", type=int, default=0, help="serve: CTAs per request launch (0: library default)")
    args = ap.parse_args()
    w = dict(WORKLOADS[args.workload])
    if args.nb:
        w["nb"] = args.nb
    if args.ib:
        w["ib"] = args.ib
    if args.variant:
        w.pop("pairs", None)
        w.pop("tree", None)
        if args.variant != "flat":
            w[args.variant] = True
    if args.slots:
        w["slots"] = args.slots
    if args.impl == "reference":
        run_reference(args, w)
    elif w.get("ls"):
        run_ls(args, w)
    elif w.get("serve"):
        run_serve(args, w)
    elif w.get("batch"):
        run_batch(args, w)
    elif w.get("qsuite"):
        run_qsuite(args, w)
    elif w.get("lu"):
        run_lu(args, w)
    else:
        run_ours(args, w)


if __name__ == "__main__":
    main()
