"""Benchmark of the FP64 TSQR hot path on GB300.

Workload: A = G diag(sigma) V^T, 4,194,304 x 64 FP64 (G iid N(0,1), sigma log-spaced
from 1 to 1e-6, V Haar orthogonal), generated on the host from fixed seeds. One step is
one pass of the whole FP64 path on that matrix: the TSQR factorization (leaf QRs and
reduction tree, sign-normalised R), the explicit thin Q, Q^T b for one right-hand side
and the least-squares solve x = R^{-1} (Q^T b)[0:n].

Metric: TSQR Gflop/s with the paper's flop counts (§4, Tables 1-2): 2mn^2 - 2n^3/3 for
R, the same again for Q, 4mnk - 2n^2k for Q^T b and n^2 k for the solve; the extra flops
of the reduction tree are not credited. Inputs (2.1 GB) are larger than L2 (129 MB).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl {ours,reference}]

With N > 1 (torchrun, one process per GPU) every rank factors its own copy of the
workload: the method has no exchange between GPUs, so this is replicas only (weak
scaling). --impl reference times the CPU oracle on a bounded row sample instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TSQR Gflop/s & %roofline (4M×64 fp64); served LSQ solves/s, p99 vs plain path"
FP64_SM_FLOPS_PER_CLK = 4.0   # 2 DFMA per clock per SM on GB300 (measured: 1.20 TFLOP/s at 2.0 GHz)
# DRAM bytes (read + write) per row of the factorization's chain launch, from an ncu
# capture of that launch (dram__bytes_read.sum + dram__bytes_write.sum at m = 1,048,576,
# n = 64, 144-row tiles: 1.050 GB); traffic grows with the rows, so it is scaled by m.
# Valid for n = 64 and that kernel build.
# end-to-end pipeline: steps rotate over this many streams, each with its own device
# buffers; the steps' kernels are ordered one after another by an event chain, so one
# step's result copy and the next steps' input copies overlap the kernels in between.
# Host-device copy bandwidth on the GB300 machines varies from run to run (a 2 GB copy takes
# 10 ms or, now and then, 30-60 ms), and more streams absorb more of that: measured at
# 4M x 64 through tsqr_qr_solve_host, on one box 84.3 / 79.9 ms per step with three streams
# against 94.4 / 86.7 / 89.8 / 90.4 with two; on another, 20 steps each, 87.2 / 92.5 /
# 85.7 / 82.1 with four against 99.7 / 97.4 / 80.7 / 87.6 with three (without the event
# chain: 89.6 with two, because concurrent steps finish together and their copies then
# queue while the GPU idles; 101.8 with one stream)
E2E_SLOTS = 4
CHAIN_DRAM_BYTES_PER_ROW_N64 = (547.427328e6 + 502.893824e6) / 1048576  # ncu, chain launch at m = 1M, n = 64


def flops_step(m, n, k=1):
    f = 2.0 * m * n * n - 2.0 * n ** 3 / 3.0
    return {"factor": f, "form_q": f, "apply_qt": 4.0 * m * n * k - 2.0 * n * n * k, "solve": float(n * n * k)}


def measured_hbm_gbs():
    """The copy bandwidth in MEASURED_PEAKS.json (written by the driver), or None."""
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
    except (OSError, ValueError, KeyError):
        return None


def rank_max(x: float, world: int, device: str) -> float:
    """The largest x over all ranks of the process group (x itself on one rank)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, t_max_ms: float) -> float:
    """Units per second of the whole job: every rank's units over the slowest rank's time."""
    return units_per_rank * world / (t_max_ms * 1e-3)


def parse(argv=None):
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--m", type=int, default=4_194_304)
    p.add_argument("--n", type=int, default=64)
    p.add_argument("--leaf-h", type=int, default=0, help="rows per leaf; 0 = the on-chip tile height")
    p.add_argument("--arity", type=int, default=2)
    p.add_argument("--tree", default="two-level", choices=["two-level", "pure"])
    p.add_argument("--cluster", type=int, default=1,
                   help="1: the binary tree's latency-bound levels in thread-block clusters (TSQR_CLUSTER)")
    p.add_argument("--decades", type=float, default=6.0)
    p.add_argument("--e2e-steps", type=int, default=20,
                   help="end-to-end steps (the pipeline's fill and drain, one input and one output "
                        "copy that nothing overlaps, are spread over them)")
    p.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-tune", action="store_true", help="skip the factorization autotuner report")
    p.add_argument("--sweep", default="", help="write a leaf-height x tree sweep (factor only) to this file")
    p.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision least-squares workload")
    p.add_argument("--no-batch", action="store_true", help="skip the batched uneven-instance workload")
    p.add_argument("--no-orth", action="store_true", help="skip the block-orthogonalization (Q-only TSQR) workload")
    p.add_argument("--no-caqr", action="store_true", help="skip the CAQR (wide matrix) workload")
    p.add_argument("--no-config2", action="store_true", help="skip the leaf-height x tree sweep and apply timings")
    p.add_argument("--caqr-only", action="store_true", help="run only the CAQR workload")
    p.add_argument("--orth-only", action="store_true", help="run only the block-orthogonalization workload")
    p.add_argument("--orth-elems", type=int, default=1 << 28, help="FP64 entries per block (m = elems / n)")
    p.add_argument("--orth-widths", default="8,16,32,64", help="block widths n, comma-separated")
    p.add_argument("--batch-count", type=int, default=10000)
    p.add_argument("--no-serve", action="store_true", help="skip the served least-squares workload")
    p.add_argument("--serve-only", action="store_true", help="run only the served least-squares workload")
    p.add_argument("--wy-min-n", type=int, default=-1,
                   help="mixed items with at least this many columns use the compact-WY 3xTF32 leaf (0: never; "
                        "-1: the library default)")
    p.add_argument("--profile-batch", type=int, default=0, metavar="N",
                   help="only run N mixed batches of 32 served-mix requests (a small case for ncu)")
    p.add_argument("--profile-chains", type=int, default=0, metavar="N",
                   help="only run N batches of 304 mixed one-chain items (4,096 x n each, R only: the "
                        "FP32 leaf chains without a tree) and report the time per column step")
    return p.parse_args(argv)


# ------------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(os.environ.get("TSQR_CLOCKS_DIR", tempfile.gettempdir()),
                                 f"tsqr_clocks_gpu{gpu_index}_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.gpu)], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return None
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for _, _, r in rows for i in range(4) if r[i].lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------- workload
def make_workload(m, n, decades):
    from paper_0912_2572_gb300 import inputs
    A = inputs.graded(m, n, decades, seed_g=0, seed_v=1)
    b = inputs.gaussian(m, 1, seed=2)
    return A, b


def dev_colmajor(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a.T)).cuda().t()


def gpu_numa_cpus(dev: int):
    """(NUMA node, CPU list) of the host node the GPU is attached to, from sysfs, or None."""
    import torch
    p = torch.cuda.get_device_properties(dev)
    bdf = f"{p.pci_domain_id:04x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0"
    try:
        node = int(open(f"/sys/bus/pci/devices/{bdf}/numa_node").read().strip())
        if node < 0:
            return None
        cpus = set()
        for part in open(f"/sys/devices/system/node/node{node}/cpulist").read().strip().split(","):
            lo, _, hi = part.partition("-")
            cpus.update(range(int(lo), int(hi or lo) + 1))
        return node, cpus
    except (OSError, ValueError):
        return None


def bind_host_to_gpu(dev: int):
    """Runs this process on the CPUs of the GPU's NUMA node, so pinned host buffers are
    allocated next to the GPU's host link (best effort; returns the node or None)."""
    found = gpu_numa_cpus(dev)
    if not found or not hasattr(os, "sched_setaffinity"):
        return None
    node, cpus = found
    allowed = cpus & os.sched_getaffinity(0)
    if not allowed:
        return None
    os.sched_setaffinity(0, allowed)
    return node


def host_pinned_colmajor(a):
    import torch
    t = torch.empty((a.shape[1], a.shape[0]), dtype=torch.float64, pin_memory=True)
    t.numpy()[:] = a.T
    return t.t()


_SIDE_STREAMS = {}


def run_step(ts, Ad, bd, b0, Q, x, leaf_h, arity, two_level, cluster=False):
    """One pass of the FP64 path; returns the factor set (caller frees). The thin Q and
    Q^T b + the solve both need only the factorization, so Q^T b runs on a second stream
    beside the thin Q (its latency-bound tree levels fill SMs the thin Q leaves idle); the
    calling stream waits for both before returning."""
    import torch
    cur = torch.cuda.current_stream()
    side = _SIDE_STREAMS.setdefault(cur.cuda_stream, torch.cuda.Stream())
    F = ts.factor(Ad, leaf_h=leaf_h, arity=arity, two_level=two_level, cluster=cluster)
    side.wait_stream(cur)
    with torch.cuda.stream(side):
        bd.copy_(b0)
        F.apply_qt(bd)
        F.solve_r(bd, X=x)
    F.form_q(Q)
    cur.wait_stream(side)
    return F


def oracle_step(oracle, A, b):
    """The oracle's pass over the same path: one Householder factorization, the thin Q,
    Q^T b and the back substitution."""
    VR, tau = oracle.householder(A)
    oracle.form_q(VR, tau)
    c = oracle.apply_qt(VR, tau, b)
    n = A.shape[1]
    return oracle.trsv_upper(np.triu(VR[:n, :n]), c[:n, 0])


def cpu_baseline(m, n, decades, budget_s=12.0):
    """The oracle as it stands on a bounded row sample: factor, thin Q, Q^T b, solve."""
    import oracle
    from paper_0912_2572_gb300 import inputs
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    oracle.set_threads(cores)
    ms_ = 32768
    while True:
        A = inputs.graded(ms_, n, decades, seed_g=0, seed_v=1)
        b = inputs.gaussian(ms_, 1, seed=2)
        t0 = time.perf_counter()
        oracle_step(oracle, A, b)
        t = time.perf_counter() - t0
        if t >= budget_s / 4 or ms_ * 2 > m:
            break
        ms_ *= 2
    fl = sum(flops_step(ms_, n).values())
    return {"value": fl / t / 1e9, "unit": "Gflop/s", "cores": cores, "kind": "oracle",
            "sample": f"{ms_} x {n} rows of the same generator (factor + thin Q + Q^T b + solve), "
                      f"{t:.2f} s"}



# ------------------------------------------------------------ extra workloads
def bench_mixed_lsq(ts):
    """Mixed-precision least squares: A 16,777,216 x 32, sigma 1..1e-4, k = 4 right-hand
    sides b = A x_true + 1e-6 N(0,1); FP32 leaves, FP64 tree, FP64 refinement. Reports the
    time of the mixed and of the FP64 solve and the error against the FP64 oracle after
    each refinement step (solving again with max_refine = 0, 1, 2, ...)."""
    import torch
    import oracle
    from paper_0912_2572_gb300 import inputs
    m, n, k = 16_777_216, 32, 4
    A = inputs.graded(m, n, 4.0, seed_g=0, seed_v=1)
    B, _ = inputs.lstsq_rhs(A, k, 1e-6, 2)
    Ad, Bd = dev_colmajor(A), dev_colmajor(B)
    leaf32 = ts.plan_describe(m, n, 1 << 20, 2, True)["tile_rows"]

    def timed(fn, reps=3):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            out = fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, out

    t_mix, (X, hist) = timed(lambda: ts.lstsq(Ad, Bd, leaf_h=512, arity=2, two_level=True, prec=ts.MIXED,
                                               max_refine=10, info=True))
    t_64, X64 = timed(lambda: ts.lstsq(Ad, Bd, leaf_h=leaf32, arity=2, two_level=True, prec=ts.FP64))
    Xo = oracle.lstsq(A, B)
    nrm = np.linalg.norm(Xo)
    steps = [h for h in hist if h > 0]
    per_step = []
    for s in range(len(steps)):
        Xs = ts.lstsq(Ad, Bd, leaf_h=512, arity=2, two_level=True, prec=ts.MIXED, max_refine=s)
        per_step.append(float(np.linalg.norm(Xs.cpu().numpy() - Xo) / nrm))
    fl = 2.0 * m * n * n - 2.0 * n ** 3 / 3.0 + 4.0 * m * n * k
    return {"workload": f"lstsq {m}x{n}, k={k}, sigma 1..1e-4 (kappa 1e4), b = A x + 1e-6 N(0,1)",
            "mixed_ms": t_mix, "fp64_ms": t_64, "speedup_vs_fp64": t_64 / t_mix,
            "mixed_err_vs_oracle": float(np.linalg.norm(X.cpu().numpy() - Xo) / nrm),
            "fp64_err_vs_oracle": float(np.linalg.norm(X64.cpu().numpy() - Xo) / nrm),
            "err_vs_oracle_per_step": per_step, "dx_over_x_per_step": steps,
            "fp64_gflops": fl / (t_64 * 1e-3) / 1e9}


def bench_block_orth(ts, peak_tflops, elems=1 << 28, widths=(8, 16, 32, 64), reps=3):
    """Q-only TSQR (tsqr_orthonormalize), the orthogonalization step of block iterative
    methods: blocks of 2^28 FP64 entries (2 GiB) at n = 8, 16, 32, 64 columns, iid N(0,1)
    drawn on the device from a seeded generator, orthonormalized out of place. Flops:
    2 (2mn^2 - 2n^3/3) (factor + thin Q). The orthogonality ||Q^T Q - I||_F is checked
    after the timed runs."""
    import torch
    out = {}
    for n in widths:
        m = elems // n
        g = torch.Generator(device="cuda")
        g.manual_seed(9000 + n)
        A = torch.randn((n, m), generator=g, dtype=torch.float64, device="cuda").t()
        Q = torch.empty((n, m), dtype=torch.float64, device="cuda").t()
        R = torch.empty((n, n), dtype=torch.float64, device="cuda").t()
        leaf_h = ts.plan_describe(m, n, 4096, 2, True)["tile_rows"]
        ts.orthonormalize(A, Q=Q, R=R, leaf_h=leaf_h, arity=2, two_level=True)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            ts.orthonormalize(A, Q=Q, R=R, leaf_h=leaf_h, arity=2, two_level=True)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        fl = 2.0 * (2.0 * m * n * n - 2.0 * n ** 3 / 3.0)
        orth = float(torch.linalg.norm(Q.t() @ Q - torch.eye(n, dtype=torch.float64, device="cuda")))
        _, prof = ts.profile_collect(lambda: ts.orthonormalize(A, Q=Q, R=R, leaf_h=leaf_h, arity=2,
                                                               two_level=True))
        torch.cuda.synchronize()
        phases = {}
        for kind, t in prof:
            phases[kind] = phases.get(kind, 0.0) + t
        out[f"n{n}"] = {"m": m, "leaf_h": leaf_h, "ms": ms, "gflops": fl / (ms * 1e-3) / 1e9,
                        "frac_of_fp64_peak": fl / (ms * 1e-3) / 1e12 / peak_tflops, "orth_err": orth,
                        "phases_ms": phases, "factor_autotune": ts.factor_autotune(A)}
        del A, Q, R
        torch.cuda.empty_cache()
    out["workload"] = ("Q-only TSQR of 2^28-entry FP64 blocks (m = 2^28 / n), iid N(0,1) from a seeded device "
                       "generator, out of place, binary two-level tree on the on-chip tile; flops 2(2mn^2 - 2n^3/3)")
    return out


def bench_caqr(ts, peak_tflops, shapes=((1 << 19, 256), (1 << 19, 512)), panels=(32, 64, 128), reps=3):
    """CAQR (tsqr_caqr, paper §2.4) of wide blocks: m = 524,288 rows, n = 256 and 512, iid
    N(0,1) from a seeded device generator; panels of 64 columns (32 and 128 timed beside
    it). Flops 2mn^2 - 2n^3/3 for the factorization and the same for the thin Q. The
    backward and orthogonality errors are checked on the device after the timed runs
    (a cuBLAS product, check only)."""
    import torch
    out = {}
    for m, n in shapes:
        g = torch.Generator(device="cuda")
        g.manual_seed(9100 + n)
        A = torch.randn((n, m), generator=g, dtype=torch.float64, device="cuda").t()
        leaf_h = ts.plan_describe(m, 64, 4096, 2, True)["tile_rows"]
        fl = 2.0 * m * n * n - 2.0 * n ** 3 / 3.0
        row = {"m": m, "n": n, "leaf_h": leaf_h}
        for panel in panels:
            ts.caqr(A, panel=panel, leaf_h=leaf_h).free()
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(reps):
                ts.caqr(A, panel=panel, leaf_h=leaf_h).free()
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            row[f"panel{panel}"] = {"factor_ms": ms, "gflops": fl / (ms * 1e-3) / 1e9,
                                    "frac_of_fp64_peak": fl / (ms * 1e-3) / 1e12 / peak_tflops}
        F = ts.caqr(A, panel=64, leaf_h=leaf_h)
        Q = F.form_q()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            F.form_q(Q)
        e1.record()
        torch.cuda.synchronize()
        qms = e0.elapsed_time(e1) / reps
        row["form_q_ms"] = qms
        row["form_q_gflops"] = fl / (qms * 1e-3) / 1e9
        _, prof = ts.profile_collect(lambda: ts.caqr(A, panel=64, leaf_h=leaf_h).free())
        torch.cuda.synchronize()
        phases = {}
        for kind, t in prof:
            phases[kind] = phases.get(kind, 0.0) + t
        row["factor_phases_ms"] = phases
        eye = torch.eye(n, dtype=torch.float64, device="cuda")
        row["orth_err"] = float(torch.linalg.norm(Q.t() @ Q - eye))
        row["backward_err"] = float(torch.linalg.norm(A - Q @ F.R) / torch.linalg.norm(A))
        F.free()
        out[f"{m}x{n}"] = row
        del A, Q
        torch.cuda.empty_cache()
    out["workload"] = ("CAQR of iid N(0,1) FP64 blocks from a seeded device generator: TSQR panels (binary "
                       "two-level tree on the on-chip tile), each panel's Q^T applied to the trailing columns; "
                       "flops 2mn^2 - 2n^3/3 (factor), the same for the thin Q")
    return out


def bench_config2(ts, Ad, m, n, leaf_h, arity, two, reps=2):
    """The leaf-height x tree sweep of the 4,194,304 x 64 matrix (factor only; the pure
    k-ary trees over leaves of h rows and the GPU two-level form, binary, 4-ary and flat),
    Q^T B at k = 1 and 4 and the thin Q for the headline configuration, and the ratio
    time(Q and R) / time(R) (paper §4, Property 1: about 2). A pure flat tree over 4M rows
    is one sequential chain on one CTA (about 17 s), so the flat tree is timed in its
    two-level form only (flat chains inside each CTA, then one flat chain over them)."""
    import torch

    def timed(fn, r=reps):
        fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(r):
            fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / r

    f_fl = 2.0 * m * n * n - 2.0 * n ** 3 / 3.0
    rows = []
    for tree in ("pure", "two-level"):
        for ar in (2, 4, 0):
            if tree == "pure" and ar == 0:
                continue
            for h in (64, 128, 256, 512, 1024):
                t = timed(lambda: ts.factor(Ad, leaf_h=h, arity=ar, two_level=tree == "two-level").free(),
                          1 if ar == 0 else reps)
                rows.append({"tree": tree, "arity": ar, "leaf_h": h, "factor_ms": t,
                             "gflops": f_fl / (t * 1e-3) / 1e9})
    F = ts.factor(Ad, leaf_h=leaf_h, arity=arity, two_level=two)
    Q = torch.empty((n, m), dtype=torch.float64, device="cuda").t()
    res = {}
    for k in (1, 4):
        B0 = torch.randn((k, m), dtype=torch.float64, device="cuda").t()
        B = B0.clone()
        t = timed(lambda: F.apply_qt(B))
        res[f"apply_qt_k{k}_ms"] = t
        res[f"apply_qt_k{k}_gflops"] = (4.0 * m * n * k - 2.0 * n * n * k) / (t * 1e-3) / 1e9
    t_q = timed(lambda: F.form_q(Q))
    t_r = timed(lambda: ts.factor(Ad, leaf_h=leaf_h, arity=arity, two_level=two).free())
    t_qr = timed(lambda: ts.factor(Ad, leaf_h=leaf_h, arity=arity, two_level=two).form_q(Q))
    F.free()
    del Q
    torch.cuda.empty_cache()
    res.update({"form_q_ms": t_q, "factor_ms": t_r, "factor_and_form_q_ms": t_qr,
                "property1_ratio_q_and_r_over_r": t_qr / t_r, "sweep": rows,
                "best": min(rows, key=lambda r: r["factor_ms"])})
    return res


def bench_batched(ts, count):
    """Batched uneven TSQR: `count` instances, m log-uniform in [256, 65536], n uniform in
    {8, 16, 32, 64}, iid N(0,1) entries (device generator, seeded), alternately FP64 and
    FP32-mixed; R of every instance. One persistent launch for the whole batch, with the
    chain length and tree arity picked by the library's autotuner (tsqr_batch_autotune) on a
    1000-instance sample;
    compared with one launch per instance (the same kernel, batches of one) and with the
    plain multi-launch tsqr_factor, both timed on a sample and reported per instance."""
    import torch
    from paper_0912_2572_gb300 import inputs
    g = inputs.rng(7)
    ms = np.exp(g.uniform(np.log(256), np.log(65536), size=count)).astype(np.int64)
    ns = g.choice([8, 16, 32, 64], size=count)
    ms = np.maximum(ms, ns)
    total = int(np.sum(ms * ns))
    gen = torch.Generator(device="cuda")
    gen.manual_seed(7)
    buf = torch.randn(total, dtype=torch.float64, device="cuda", generator=gen)
    items = []
    off = 0
    for q in range(count):
        m, n = int(ms[q]), int(ns[q])
        A = buf[off:off + m * n].view(n, m).t()
        off += m * n
        items.append({"A": A, "prec": q & 1})
    flops = float(np.sum(2.0 * ms * ns * ns - 2.0 * ns ** 3 / 3.0))

    def run(its, L, ar, reps=1):
        ts.batch_solve(its, chain_tiles=L, arity=ar)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            ts.batch_solve(its, chain_tiles=L, arity=ar)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    # the library's autotuner times every (chain length, arity) on the first 1000 items
    L_best, ar_best, table = ts.batch_autotune(items, sample=min(1000, count))
    tune = {f"L{L}_a{ar}": ms for (L, ar), ms in table.items()}
    t_batch = run(items, L_best, ar_best, reps=2)
    # the same batch planned once and replayed as a CUDA graph
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plan = ts.BatchPlan(items, chain_tiles=L_best, arity=ar_best)
    t_plan = time.perf_counter() - t0
    plan.run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(3):
        plan.run()
    e1.record()
    torch.cuda.synchronize()
    t_replay = e0.elapsed_time(e1) / 3
    plan_status, _ = plan.results()
    plan.close()
    # one launch per instance and the plain API, on the first 500 instances
    few = items[:min(500, count)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for it in few:
        ts.batch_solve([it], chain_tiles=L_best, arity=ar_best)
    torch.cuda.synchronize()
    t_one = (time.perf_counter() - t0) / len(few)
    t0 = time.perf_counter()
    for it in few:
        A = it["A"]
        h = max(A.shape[1], 256)
        ts.factor(A, leaf_h=h, arity=2, two_level=True).free()
    torch.cuda.synchronize()
    t_plain = (time.perf_counter() - t0) / len(few)
    return {"workload": f"{count} instances, m log-uniform [256, 65536], n in {{8,16,32,64}}, half FP64 / half "
                        "FP32-mixed, R of each",
            "autotune_ms_on_1000": tune, "chain_tiles": L_best, "arity": ar_best,
            "batched_ms": t_batch, "batched_instances_per_s": count / (t_batch * 1e-3),
            "batched_gflops": flops / (t_batch * 1e-3) / 1e9,
            "plan_create_s": t_plan, "graph_replay_ms": t_replay,
            "graph_replay_instances_per_s": count / (t_replay * 1e-3),
            "graph_replay_gflops": flops / (t_replay * 1e-3) / 1e9,
            "graph_replay_failed": sum(1 for x in plan_status if x != 0),
            "one_launch_per_instance_instances_per_s": 1.0 / t_one,
            "plain_tsqr_factor_instances_per_s": 1.0 / t_plain,
            "speedup_vs_one_launch_per_instance": t_one * count / (t_batch * 1e-3),
            "speedup_vs_plain": t_plain * count / (t_batch * 1e-3)}

def ts_plan_rows(m, n, nc):
    import paper_0912_2572_gb300 as ts
    return ts.plan_describe(m, n, 1 << 20, 2, True, nc=nc)["tile_rows"]


def make_served_pool(count, seed=11):
    """Least-squares requests shaped like the served workload: m log-uniform in [1e3, 1e6],
    n uniform over {16, 32, 64, 128}, k uniform in 1..8, A = G diag(sigma) V^T with G iid
    N(0,1) (device generator), sigma log-spaced from 1 to 1/kappa with kappa log-uniform in
    [1, 1e4], V Haar-orthogonal, and b = A x_true + 1e-6 N(0,1). Built on the device."""
    import torch
    from paper_0912_2572_gb300 import inputs
    g = inputs.rng(seed)
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    pool = []
    for q in range(count):
        m = int(np.exp(g.uniform(np.log(1e3), np.log(1e6))))
        n = int(g.choice([16, 32, 64, 128]))
        k = int(g.integers(1, 9))
        dec = float(g.uniform(0.0, 4.0))
        sig = torch.tensor(inputs.log_spectrum(n, dec), device="cuda")
        V = torch.tensor(inputs.haar_orthogonal(n, seed * 100003 + q), device="cuda")
        G = torch.randn((n, m), dtype=torch.float64, device="cuda", generator=gen).t()
        A = torch.empty((n, m), dtype=torch.float64, device="cuda").t()
        A.copy_(G * sig @ V.t())
        del G
        xt = torch.randn((n, k), dtype=torch.float64, device="cuda", generator=gen)
        B = torch.empty((k, m), dtype=torch.float64, device="cuda").t()
        B.copy_(A @ xt + 1e-6 * torch.randn((m, k), dtype=torch.float64, device="cuda", generator=gen))
        nc = n + k if n + k <= 128 else n  # the plain path fuses Q^T B when it fits
        leaf_h = ts_plan_rows(m, n, nc)
        pool.append({"A": A, "B": B, "m": m, "n": n, "k": k, "kappa": 10.0 ** dec, "leaf_h": leaf_h})
    return pool


def bench_served(ts, pool_size=160, rate=2000.0, arrivals=2000, closed=800, plain_sample=96, streams=2,
                 max_batch=128, seed=11):
    """Served least squares: a continuous-batching server fed (a) open-loop by a Poisson
    stream at `rate` requests/s and (b) closed-loop with `closed` requests at once
    (saturation throughput); compared with the plain path, one tsqr_lstsq FP64 call per
    request in sequence, synchronised after each. Requests cycle through a pool of
    `pool_size` distinct device-resident problems; latencies are from submission to the
    server's observation of completion. Each X is checked against the plain path."""
    import torch
    pool = make_served_pool(pool_size, seed)
    torch.cuda.synchronize()
    g = np.random.Generator(np.random.PCG64(seed + 1))

    def lsq_flops(r):
        m, n, k = r["m"], r["n"], r["k"]
        return 2.0 * m * n * n - 2.0 * n ** 3 / 3.0 + 4.0 * m * n * k

    # plain path: one request at a time through tsqr_lstsq (FP64, fused Q^T B when n + k <= 128)
    for r in pool[:4]:
        ts.lstsq(r["A"], r["B"], leaf_h=r["leaf_h"], arity=2, two_level=True, prec=ts.FP64)
    torch.cuda.synchronize()
    order = [int(i) for i in g.integers(0, pool_size, size=plain_sample)]
    t0 = time.perf_counter()
    Xplain = {}
    for i in order:
        Xplain[i] = ts.lstsq(pool[i]["A"], pool[i]["B"], leaf_h=pool[i]["leaf_h"], arity=2, two_level=True,
                             prec=ts.FP64)
        torch.cuda.synchronize()
    t_plain = (time.perf_counter() - t0) / plain_sample
    plain_fl = float(np.mean([lsq_flops(pool[i]) for i in order]))

    def submit_all(srv, idx, prec, times=None):
        outs = {}
        start = time.perf_counter()
        for j, i in enumerate(idx):
            if times is not None:
                while time.perf_counter() - start < times[j]:
                    pass
            t, (_, X) = srv.submit({"A": pool[i]["A"], "B": pool[i]["B"], "want_r": False, "prec": prec})
            outs[t] = (i, X)
        return outs

    def collect(srv, n_expected, limit_s=300.0):
        done = []
        t_end = time.perf_counter() + limit_s
        while len(done) < n_expected:
            done += srv.poll()
            if time.perf_counter() > t_end:
                raise RuntimeError(f"served requests incomplete after {limit_s} s: {len(done)}/{n_expected}")
            time.sleep(0.0002)
        return done

    def server(resident):
        if resident:  # one persistent kernel admitting requests while it runs
            return ts.Server(resident=True, chain_tiles=8, idle_us=20_000)
        return ts.Server(max_batch=max_batch, streams=streams, chain_tiles=8)

    def closed_loop(prec, resident=False):
        with server(resident) as srv:
            warm = [int(i) for i in g.integers(0, pool_size, size=64)]
            submit_all(srv, warm, prec)
            collect(srv, len(warm))
            b0 = srv.stats()["launches" if resident else "batches"]
            idx = [int(i) for i in g.integers(0, pool_size, size=closed)]
            t0 = time.perf_counter()
            outs = submit_all(srv, idx, prec)
            done = collect(srv, closed)
            t = time.perf_counter() - t0
            st = srv.stats()
        lat = np.array([d[1] for d in done])
        errs = [float(torch.linalg.norm(X - Xplain[i]) / torch.linalg.norm(Xplain[i]))
                for i, X in outs.values() if i in Xplain]
        out = {"requests": closed, "solves_per_s": closed / t,
               "gflops_fp64_equiv": sum(lsq_flops(pool[i]) for i in idx) / t / 1e9,
               "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
               "failed": sum(1 for d in done if d[2] != 0),
               "max_rel_diff_vs_plain_fp64": max(errs) if errs else None}
        if resident:
            out.update({"launches": st["launches"] - b0, "most_in_flight": st["max_in_flight"]})
        else:
            out.update({"batches": st["batches"] - b0, "largest_batch": st["max_batch"]})
        return out

    res = {"closed_loop": {}}
    for name, prec in (("fp64", ts.FP64), ("auto", ts.AUTO), ("mixed", ts.MIXED)):
        res["closed_loop"][name] = closed_loop(prec)
    best = max(res["closed_loop"], key=lambda n: res["closed_loop"][n]["solves_per_s"])
    prec = {"fp64": ts.FP64, "auto": ts.AUTO, "mixed": ts.MIXED}[best]
    # open loop: Poisson arrivals at `rate`
    with ts.Server(max_batch=max_batch, streams=streams, chain_tiles=8) as srv:
        warm = [int(i) for i in g.integers(0, pool_size, size=64)]
        submit_all(srv, warm, prec)
        collect(srv, len(warm))
        b0 = srv.stats()["batches"]
        gaps = g.exponential(1.0 / rate, size=arrivals)
        times = np.cumsum(gaps) - gaps[0]
        idx = [int(i) for i in g.integers(0, pool_size, size=arrivals)]
        t0 = time.perf_counter()
        submit_all(srv, idx, prec, times)
        t_sub = time.perf_counter() - t0
        done = collect(srv, arrivals)
        t_open = time.perf_counter() - t0
        lat = np.array([d[1] for d in done])
        res["open_loop"] = {"prec": best, "offered_per_s": rate, "arrivals": arrivals, "submit_span_s": t_sub,
                            "completed_per_s": arrivals / t_open,
                            "p50_ms": float(np.percentile(lat, 50) * 1e3),
                            "p99_ms": float(np.percentile(lat, 99) * 1e3),
                            "batches": srv.stats()["batches"] - b0,
                            "failed": sum(1 for d in done if d[2] != 0)}
    # the plain path under Poisson arrivals: one request at a time, first come first
    # served; latency from arrival to completion
    def plain_open_loop(rate_, count):
        gaps_ = g.exponential(1.0 / rate_, size=count)
        arr = np.cumsum(gaps_) - gaps_[0]
        ids = [int(i) for i in g.integers(0, pool_size, size=count)]
        lat_ = []
        start = time.perf_counter()
        for a, i in zip(arr, ids):
            while time.perf_counter() - start < a:
                pass
            ts.lstsq(pool[i]["A"], pool[i]["B"], leaf_h=pool[i]["leaf_h"], arity=2, two_level=True, prec=ts.FP64)
            torch.cuda.synchronize()
            lat_.append(time.perf_counter() - start - a)
        lat_ = np.array(lat_)
        return {"offered_per_s": rate_, "arrivals": count, "completed_per_s": count / (time.perf_counter() - start),
                "p50_ms": float(np.percentile(lat_, 50) * 1e3), "p99_ms": float(np.percentile(lat_, 99) * 1e3)}

    def served_open_loop(rate_, count, prec_, resident=False):
        with server(resident) as srv:
            warm = [int(i) for i in g.integers(0, pool_size, size=32)]
            submit_all(srv, warm, prec_)
            collect(srv, len(warm))
            gaps_ = g.exponential(1.0 / rate_, size=count)
            times_ = np.cumsum(gaps_) - gaps_[0]
            idx_ = [int(i) for i in g.integers(0, pool_size, size=count)]
            t0_ = time.perf_counter()
            submit_all(srv, idx_, prec_, times_)
            done_ = collect(srv, count)
            t_ = time.perf_counter() - t0_
        lat_ = np.array([d[1] for d in done_])
        return {"offered_per_s": rate_, "arrivals": count, "completed_per_s": count / t_,
                "p50_ms": float(np.percentile(lat_, 50) * 1e3), "p99_ms": float(np.percentile(lat_, 99) * 1e3)}

    res["plain_open_loop"] = plain_open_loop(rate, 300)
    res["low_rate_200_per_s"] = {"plain": plain_open_loop(200.0, 300), "served": served_open_loop(200.0, 300, prec)}
    # the resident server (requests admitted into the running persistent kernel), MIXED
    res["resident"] = {"closed_loop_mixed": closed_loop(ts.MIXED, resident=True),
                       "open_loop_2000_per_s": served_open_loop(rate, arrivals, ts.MIXED, resident=True),
                       "open_loop_200_per_s": served_open_loop(200.0, 300, ts.MIXED, resident=True),
                       "launching_server_open_loop_200_per_s_mixed": served_open_loop(200.0, 300, ts.MIXED)}
    res["plain_fp64"] = {"solves_per_s": 1.0 / t_plain, "ms_per_solve": t_plain * 1e3,
                         "gflops": plain_fl / t_plain / 1e9, "sample": plain_sample}
    res["speedup_closed_vs_plain"] = {k: v["solves_per_s"] / res["plain_fp64"]["solves_per_s"]
                                      for k, v in res["closed_loop"].items()}
    res["workload"] = (f"lstsq requests: m log-uniform [1e3, 1e6], n in {{16,32,64,128}}, k 1..8, kappa "
                       f"log-uniform [1, 1e4], b = A x + 1e-6 N(0,1); pool of {pool_size} device-resident "
                       f"problems; server: {streams} streams, <= {max_batch} per launch")
    del pool
    torch.cuda.empty_cache()
    return res


# ------------------------------------------------------------------ reference
def bench_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    from paper_0912_2572_gb300 import inputs
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count()
    oracle.set_threads(cores)
    ms_ = 65536
    A = inputs.graded(ms_, args.n, args.decades, seed_g=0, seed_v=1)
    b = inputs.gaussian(ms_, 1, seed=2)

    def step():
        oracle_step(oracle, A, b)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    t = time.perf_counter() - t0
    fl = sum(flops_step(ms_, args.n).values())
    val = fl * args.steps / t / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "Gflop/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"tsqr_fp64 {args.m}x{args.n} graded (sigma 1..1e-{args.decades:g}); "
                                   f"reference = CPU oracle on a {ms_}-row sample per step"},
            "cpu_baseline": {"value": val, "unit": "Gflop/s", "cores": cores, "kind": "oracle",
                             "sample": f"{ms_} x {args.n} rows per step (factor + thin Q + Q^T b + solve)"},
            "e2e": {"value": val, "unit": "Gflop/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------- ours
def sweep(args, ts, Ad, path):
    import torch
    rows = []
    for tree in ("pure", "two-level"):
        for arity in (2, 4, 0):
            for h in (64, 128, 256, 512, 1024):
                if tree == "pure" and arity == 0 and h < 1024:
                    continue  # a flat tree is one sequential chain: one point is enough
                two = tree == "two-level"
                for _ in range(1):
                    F = ts.factor(Ad, leaf_h=h, arity=arity, two_level=two)
                    F.free()
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                reps = 1 if (arity == 0 and not two) else 3
                e0.record()
                for _ in range(reps):
                    F = ts.factor(Ad, leaf_h=h, arity=arity, two_level=two)
                    F.free()
                e1.record()
                torch.cuda.synchronize()
                t = e0.elapsed_time(e1) / reps
                g = flops_step(args.m, args.n)["factor"] / (t * 1e-3) / 1e9
                rows.append({"tree": tree, "arity": arity, "leaf_h": h, "ms": t, "gflops": g})
                print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    with open(path, "w") as f:
        for r in rows:
            f.write(json.dumps(r) + "\n")


def bench_ours(args):
    import torch
    import torch.distributed as dist
    import paper_0912_2572_gb300 as ts
    from paper_0912_2572_gb300 import build as tsbuild

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    all_cpus = os.sched_getaffinity(0) if hasattr(os, "sched_getaffinity") else None
    numa = bind_host_to_gpu(local)
    if not os.path.exists(os.path.join(ROOT, "paper_0912_2572_gb300", "libtsqr.so")) and rank == 0:
        tsbuild.build()
    if world > 1:
        dist.barrier()
    if args.wy_min_n >= 0:
        ts.set_mixed_wy_min_n(args.wy_min_n)
    if args.serve_only:
        if rank == 0:
            print(json.dumps({"served": bench_served(ts)}), flush=True)
        return 0
    if args.orth_only:
        if rank == 0:
            widths = tuple(int(w) for w in args.orth_widths.split(","))
            print(json.dumps({"block_orth": bench_block_orth(ts, ts.probe_fp64_peak(), args.orth_elems, widths)}),
                  flush=True)
        return 0
    if args.caqr_only:
        if rank == 0:
            print(json.dumps({"caqr": bench_caqr(ts, ts.probe_fp64_peak())}), flush=True)
        return 0
    if args.profile_batch:
        pool = make_served_pool(32, 11)
        items = [{"A": r["A"], "B": r["B"], "want_r": False, "prec": ts.MIXED} for r in pool]
        for _ in range(args.profile_batch):
            ts.batch_solve(items, chain_tiles=8)
        torch.cuda.synchronize()
        _, prof = ts.profile_collect(lambda: ts.batch_solve(items, chain_tiles=8))
        rows = sum(r["m"] for r in pool)
        print(json.dumps({"profile_batch": {"requests": len(pool), "rows": rows,
                                            "phases_ms": {k: ms for k, ms in prof}}}), flush=True)
        return 0

    if args.profile_chains:
        # one chain of 32 tiles of 128 rows per item, two CTAs per SM on every SM: the FP32
        # column step's latency with the GPU full, with no FP64 tree above the chains
        n, count = args.n, 2 * torch.cuda.get_device_properties(local).multi_processor_count
        gen = torch.Generator(device="cuda")
        gen.manual_seed(5)
        items = [{"A": torch.randn((n, 4096), dtype=torch.float64, device="cuda", generator=gen).t(),
                  "prec": ts.MIXED} for _ in range(count)]
        for _ in range(args.profile_chains):
            ts.batch_solve(items)
        torch.cuda.synchronize()
        _, prof = ts.profile_collect(lambda: ts.batch_solve(items))
        ms = sum(t for k, t in prof if k == "batch")
        print(json.dumps({"profile_chains": {"items": count, "m": 4096, "n": n, "batch_ms": ms,
                                             "us_per_column_step": ms * 1e3 / (32 * n)}}), flush=True)
        return 0

    m, n = args.m, args.n
    two = args.tree == "two-level"
    cl = bool(args.cluster) and args.arity == 2
    leaf_h = args.leaf_h or ts.plan_describe(m, n, 4096, args.arity, two)["tile_rows"]
    A, b = make_workload(m, n, args.decades)
    Ad = dev_colmajor(A)
    bd = dev_colmajor(b)
    b0 = bd.clone()
    Q = torch.empty((n, m), dtype=torch.float64, device="cuda").t()
    x = torch.empty((1, n), dtype=torch.float64, device="cuda").t()
    fl = flops_step(m, n)
    fl_step = sum(fl.values())

    if args.sweep and rank == 0:
        sweep(args, ts, Ad, args.sweep)

    for _ in range(args.warmup):
        run_step(ts, Ad, bd, b0, Q, x, leaf_h, args.arity, two, cl).free()
    torch.cuda.synchronize()
    info = ts.factor(Ad, leaf_h=leaf_h, arity=args.arity, two_level=two, cluster=cl)
    plan = info.info()
    info.free()
    torch.cuda.synchronize()

    # --- timed region: K steps, CUDA events on the launching stream, launch profile live
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        def timed():
            ev0.record(stream)
            for _ in range(args.steps):
                run_step(ts, Ad, bd, b0, Q, x, leaf_h, args.arity, two, cl).free()
            ev1.record(stream)
            torch.cuda.synchronize()
        _, prof = ts.profile_collect(timed)
    if world > 1:
        dist.barrier()
    t_ms = ev0.elapsed_time(ev1)
    t_max = rank_max(t_ms, world, "cuda")
    value = whole_job_rate(fl_step * args.steps, world, t_max) / 1e9

    # --- per-phase times from the launch profile
    phase_ms = {}
    for kind, ms in prof:
        phase_ms[kind] = phase_ms.get(kind, 0.0) + ms
    chain = [ms for kind, ms in prof if kind == "factor_chains"]
    chain_ms = sum(chain) / max(1, len(chain))
    # chain launch algorithmic flops: every chain is a Householder QR of its own rows
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    if two:
        n_chains = min(plan["leaves"], sms * plan["ctas_per_sm"] * 4)
    else:
        n_chains = 1 if args.arity == 0 else plan["leaves"]
    chain_flops = 2.0 * m * n * n - n_chains * 2.0 * n ** 3 / 3.0
    achieved = chain_flops / (chain_ms * 1e-3) / 1e12
    clocks = clk.summary()
    peak_derived = sms * FP64_SM_FLOPS_PER_CLK * 2.070e9 / 1e12
    peak_measured, probe_mhz = ts.probe_fp64_peak(clock=True)  # after the timed region
    dmma_tflops, dmma_mhz = ts.probe_dmma_peak(clock=True)      # FP64 tensor cores, for comparison
    peak = peak_measured if peak_measured > 0 else peak_derived
    factor_ms = (phase_ms.get("factor_chains", 0) + phase_ms.get("factor_tree", 0)) / args.steps

    # --- end to end through the library's host-buffer call (tsqr_qr_solve_host): every
    # step copies A and b from pinned host memory to the device, runs the whole path, and
    # copies Q, R and x back, all inside the timed region. Steps rotate over E2E_SLOTS
    # streams; each call's kernels wait (its `after` event) for the previous call's kernels,
    # so one step's copies overlap the neighbouring steps' kernels.
    e2e = None
    if not args.no_e2e:
        # the pinned outputs first and the inputs last, right before the loop: on the GB300
        # box the host-to-device bandwidth from a pinned buffer decays in the seconds after
        # it was written (210 -> 145 GB/s in 20 s idle, and lower right after other large
        # pinned allocations), so the copy bandwidth is also measured just before the loop
        slots = []
        for q in range(E2E_SLOTS):
            ev = torch.cuda.Event()
            ev.record(stream)  # materialise the event handle
            slots.append({"s": torch.cuda.Stream(), "ev": ev,
                          "Qh": torch.empty((n, m), dtype=torch.float64, pin_memory=True).t(),
                          "Rh": torch.empty((n, n), dtype=torch.float64, pin_memory=True).t(),
                          "xh": torch.empty((1, n), dtype=torch.float64, pin_memory=True).t(),
                          "st": torch.zeros(1, dtype=torch.int32).pin_memory()})
        torch.cuda.synchronize()
        Ah = host_pinned_colmajor(A)
        bh = host_pinned_colmajor(b)
        probe = torch.empty_like(Ad)
        p0, p1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        p0.record(stream)
        probe.copy_(Ah, non_blocking=True)
        p1.record(stream)
        torch.cuda.synchronize()
        h2d_before = 8.0 * m * n / (p0.elapsed_time(p1) * 1e-3) / 1e9
        del probe
        done = [None]

        def e2e_step(i):
            sl = slots[i % E2E_SLOTS]
            ts.qr_solve_host(Ah, bh, Q=sl["Qh"], R=sl["Rh"], X=sl["xh"], status=sl["st"], leaf_h=leaf_h,
                             arity=args.arity, two_level=two, cluster=cl, stream=sl["s"], after=done[0],
                             done=sl["ev"])
            done[0] = sl["ev"]

        # one untimed pass per stream (each stream's first allocations grow the pool)
        for i in range(E2E_SLOTS):
            e2e_step(i)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as e2e_clk:
            e0.record(stream)
            for sl in slots:
                sl["s"].wait_event(e0)
            for i in range(args.e2e_steps):
                e2e_step(i)
            for sl in slots:
                stream.wait_stream(sl["s"])
            e1.record(stream)
            torch.cuda.synchronize()
        te = rank_max(e0.elapsed_time(e1), world, "cuda")
        e2e = {"value": whole_job_rate(fl_step * args.e2e_steps, world, te) / 1e9, "unit": "Gflop/s",
               "h2d_bytes_per_step": 8 * (m * n + m), "d2h_bytes_per_step": 8 * (m * n + n * n + n),
               "ms_per_step": te / args.e2e_steps, "pipelined_streams": E2E_SLOTS,
               "api": "tsqr_qr_solve_host (host buffers, copies inside the call)",
               "clocks": e2e_clk.summary()}
        last = slots[(args.e2e_steps - 1) % E2E_SLOTS]
        xe = last["xh"].numpy()[:, 0]
        xd = x.cpu().numpy()[:, 0]
        e2e["x_rel_diff_vs_device_run"] = float(np.linalg.norm(xe - xd) / np.linalg.norm(xd))
        e2e["status"] = int(last["st"][0])
        # this box's pinned-copy bandwidth, after the timed region (the e2e figure depends on it)
        Qd = torch.empty((n, m), dtype=torch.float64, device="cuda").t()
        Ad2 = torch.empty_like(Ad)
        c0, c1, c2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        c0.record(stream)
        Ad2.copy_(Ah, non_blocking=True)
        c1.record(stream)
        last["Qh"].copy_(Qd, non_blocking=True)
        c2.record(stream)
        torch.cuda.synchronize()
        e2e["copy_gbs"] = {"h2d_before": h2d_before, "h2d": 8.0 * m * n / (c0.elapsed_time(c1) * 1e-3) / 1e9,
                           "d2h": 8.0 * m * n / (c1.elapsed_time(c2) * 1e-3) / 1e9}
        del Ah, slots, Qd, Ad2

    # the library's factorization autotuner on the same matrix (leaf height x arity x tree
    # form, factor only); reported beside the headline's fixed configuration
    tuned = None
    if rank == 0 and not args.no_tune:
        tuned = ts.factor_autotune(Ad)
        tuned["headline_factor_ms"] = factor_ms

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        if all_cpus:
            os.sched_setaffinity(0, all_cpus)  # the oracle baseline uses every host core
        cpu = cpu_baseline(m, n, args.decades)
    del Q
    config2 = None if args.no_config2 or rank != 0 else bench_config2(ts, Ad, m, n, leaf_h, args.arity, two)
    torch.cuda.empty_cache()
    caqr = None if args.no_caqr or rank != 0 else bench_caqr(ts, peak)
    torch.cuda.empty_cache()
    mixed = None if args.no_mixed or rank != 0 else bench_mixed_lsq(ts)
    torch.cuda.empty_cache()
    block_orth = None if args.no_orth or rank != 0 else bench_block_orth(
        ts, peak, args.orth_elems, tuple(int(w) for w in args.orth_widths.split(",")))
    torch.cuda.empty_cache()
    batched = None if args.no_batch or rank != 0 else bench_batched(ts, args.batch_count)
    torch.cuda.empty_cache()
    served = None if args.no_serve or rank != 0 else bench_served(ts)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "Gflop/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"tsqr_fp64 {m}x{n} A=G*diag(sigma)*V^T, sigma 1..1e-{args.decades:g}; "
                                   "step = factor + thin Q + Q^T b + solve",
                       "m": m, "n": n, "leaf_h": leaf_h, "arity": args.arity, "tree": args.tree,
                       "cluster_tier": cl,
                       "tile_rows": plan["tile_rows"], "chains": n_chains, "ctas_per_sm": plan["ctas_per_sm"],
                       "l2": "inputs (2.1 GB) larger than L2, no flush", "parallelism": f"replicas x{world}",
                       "host_numa_node": numa},
            "phases": {"factor_ms": factor_ms,
                       "factor_gflops": fl["factor"] / (factor_ms * 1e-3) / 1e9 if factor_ms else None,
                       "form_q_ms": phase_ms.get("form_q", 0) / args.steps,
                       # Q^T b runs beside the thin Q on a second stream: its launches' event
                       # times include the time they wait for SMs (alone: config2.apply_qt_k1_ms)
                       "apply_qt_ms_beside_form_q": phase_ms.get("apply_qt", 0) / args.steps,
                       "small_ms": phase_ms.get("small", 0) / args.steps},
            "roofline": {"kernel": "k_factor (leaf/flat-chain launch)", "bound": "alu", "achieved": achieved,
                         "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                         "traffic": (CHAIN_DRAM_BYTES_PER_ROW_N64 * m if n == 64 else None),
                         "hbm_gbs": (CHAIN_DRAM_BYTES_PER_ROW_N64 * m / (chain_ms * 1e-3) / 1e9 if n == 64 else None),
                         "hbm_peak_gbs": measured_hbm_gbs(),
                         "peak_source": "measured" if peak_measured > 0 else "derived",
                         "peak_note": f"FP64 DFMA measured live by tsqr_probe_fp64_peak (independent DFMA chains "
                                      f"on every SM): {peak_measured:.3f} TFLOP/s at {probe_mhz:.0f} MHz; derived {sms} SMs x "
                                      f"{FP64_SM_FLOPS_PER_CLK} flop/clk x 2.07 GHz = {peak_derived:.3f}; the "
                                      "measured-peaks file has no FP64 entry",
                         "frac_of_derived": achieved / peak_derived,
                         "fp64_tensor_tflops_measured": dmma_tflops,
                         "fp64_tensor_note": f"DMMA (mma.sync m8n8k4 FP64, tsqr_probe_dmma_peak): {dmma_tflops:.3f} "
                                             f"TFLOP/s at {dmma_mhz:.0f} MHz against the FMA pipe's "
                                             f"{peak_measured:.3f}: the FP64 path stays on the FMA pipe"},
            "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": len(prof), "clocks": clocks,
            "factor_autotune": tuned, "config2": config2, "caqr": caqr, "mixed_lsq": mixed,
            "block_orth": block_orth, "batched": batched,
            "served": served,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return bench_reference(args)
    return bench_ours(args)


if __name__ == "__main__":
    sys.exit(main())
