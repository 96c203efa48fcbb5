#!/usr/bin/env python
"""Benchmark: quantum-kernel Gram entries/s on one GB300 (or G GPUs, weak scaling).

Workload (default): n = 784 qubits (28 x 28 MNIST-like features, 80 % exact zeros,
the rest uniform on (0, 1] * pi; seed 4), reps = 2 (bond dimension 4),
N = 8192 points, the full symmetric 8192 x 8192 Gram.  One step = the whole hot
path: MPS build from the feature matrix (FP64, gate by gate; in split FP32 at reps = 2 stored
as the two gauged phases of every site) + the all-pairs contraction over the upper-triangle tiles
(diagonal included) + the mirror write.  Entries counted = unique pairs
contracted, N (N + 1) / 2 per step.

Timing: W untimed warm-up steps, then K steps, each bracketed by CUDA events on
the launching stream with a synchronize on both sides; the L2 (129 MB) is
flushed by writing a 512 MB buffer between timed steps.  Under torchrun with G
ranks the Gram grows to round(N sqrt(G)) points (same distribution and seed), so
each rank's contiguous, pair-balanced share of its tiles stays the size of the
one-GPU Gram (weak scaling, no collective on the data path); the time is the max
over ranks and the value counts the pairs of all ranks.

--impl reference times the CPU oracle (plain FP64 C, closed-form MPS overlap,
OpenMP over pairs) on the host cores on a bounded random sample of the same
workload's pairs, and prints the same JSON line with "impl": "reference".
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2405_02630_gb300 import inputs  # noqa: E402

MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
N_SM = 152
FP32_LANES_PER_SM = 128
SM_MAX_MHZ_NOMINAL = 2070.0


def structured_cmacs_per_entry(n: int, reps: int) -> int:
    """Complex MACs per kernel entry with minimal bonds b_k = min(2^reps, 2^k, 2^(n-k)),
    counting only the nonzero blocks (the diagonal last layer makes a quarter of the
    dense 2 b_l b_r (b_l + b_r) per site necessary)."""
    b = [1] + [min(2 ** reps, 2 ** k, 2 ** (n - k)) for k in range(1, n)] + [1]
    dense = sum(2 * b[k] * b[k + 1] * (b[k] + b[k + 1]) for k in range(n))
    return dense // 4


def factorized_cmacs_per_entry(n: int, reps: int, prec: str = "fp64") -> int:
    """Complex MACs per kernel entry of the contraction as the kernels carry it out.
    Block form (reps 1, 3): per site rho = r(i) conj(r(j)) (1), G_s = E_0 + rho_s E_1
    (chi^2/2), X_s = a_0s^T G_s and E'_s = X_s conj(b_0s) (chi^3/4 each), bonds padded to chi.
    Phase form (reps 2, plain FP32): rho (1), G (8), X and E' with the unit entries of a and b
    added rather than multiplied (12 each): 33.  Gauged form (FP64 and split FP32), n + 1 sites
    (one virtual): reps 2, two phase products, Y (8), X (8), E' (8): 26 per site; reps 3, the
    Kronecker stages Z, Y (32 each), the mix (32), W, E' (32 each) and two phase products: 162."""
    chi = 2 ** reps
    if prec in ("fp32_split", "fp64") and reps in (2, 3):
        return (n + 1) * (26 if reps == 2 else 162)
    if reps == 2:
        return n * 33
    return n * (chi ** 3 // 2 + chi ** 2 // 2 + 1)


def dense_cmacs_per_entry(n: int, reps: int) -> int:
    b = [1] + [min(2 ** reps, 2 ** k, 2 ** (n - k)) for k in range(1, n)] + [1]
    return sum(2 * b[k] * b[k + 1] * (b[k] + b[k + 1]) for k in range(n))


# real FP32 FMAs each arithmetic issues per complex MAC of the contraction
FMA_PER_CMAC = {"fp32": 4, "fp32_split": 12, "fp64": 4}

# DRAM bytes (read + write) of one pair-kernel launch, from one ncu capture of the
# same workload, precision and pipeline configuration (dram__bytes_read.sum +
# dram__bytes_write.sum, one pass over the full-size launch), each stored with the
# digest of the kernel sources it was captured on (kernel_digest()).  A workload or
# configuration not captured, or captured on other kernel sources, reports null.
MEASURED_TRAFFIC_BYTES = {
    ("gram_n784_r2_N8192", "fp32_split", 9): ("e5bc5932b71cb763", 2_660_363_776 + 550_344_448),
    ("cfg4_n784_r3_N8192", "fp32_split", 20): ("e5bc5932b71cb763", 4_014_598_400 + 567_146_240),
}
KERNEL_SOURCES = ("pair_contract.cuh", "pair_contract.cu", "qsvm_common.cuh")


def kernel_digest() -> str:
    """sha256 (first 16 hex digits) of the pair-kernel sources."""
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2405_02630_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(workload: str, prec: str, config: int):
    entry = MEASURED_TRAFFIC_BYTES.get((workload, prec, config))
    if entry is None or entry[0] != kernel_digest():
        return None
    return entry[1]


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = [r.split(",") for r in open(self.path).read().strip().splitlines() if r.strip()]
        os.unlink(self.path)
        sm, smax, power, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                smax.append(float(r[2]))
                power.append(float(r[3]))
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "power_w_max": max(power) if power else None, "reasons": sorted(reasons)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def cpu_oracle_rate(X, reps, n_pairs, seed, threads=0):
    """Times the CPU oracle on n_pairs random pairs of X (upper triangle incl. diagonal)."""
    from oracle import oracle
    rng = np.random.default_rng(seed)
    N = X.shape[0]
    a = rng.integers(0, N, n_pairs)
    b = rng.integers(0, N, n_pairs)
    ia, ib = np.minimum(a, b), np.maximum(a, b)
    t0 = time.perf_counter()
    oracle.mps_pairs(X, X, ia, ib, reps, threads=threads)
    dt = time.perf_counter() - t0
    return n_pairs / dt, dt


def gemm_peaks(dev):
    """Library GEMM throughput on this GPU, as a measured ceiling beside the derived
    FP32 peak: torch.matmul float64 4096^3 and float32 (TF32 off) 8192^3, best of 3
    after one warm-up, CUDA events, TFLOP/s at 2 n^3."""
    import torch
    out = {}
    tf32 = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        for name, dt, m in (("f64", torch.float64, 4096), ("f32", torch.float32, 8192)):
            a = torch.randn(m, m, dtype=dt, device=dev)
            b = torch.randn(m, m, dtype=dt, device=dev)
            c = torch.empty(m, m, dtype=dt, device=dev)
            torch.matmul(a, b, out=c)
            best = float("inf")
            for _ in range(3):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b, out=c)
                e1.record()
                torch.cuda.synchronize(dev)
                best = min(best, e0.elapsed_time(e1))
            out[name] = 2.0 * m ** 3 / (best * 1e-3) / 1e12
            del a, b, c
    finally:
        torch.backends.cuda.matmul.allow_tf32 = tf32
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import oracle
    oracle.build()
    if args.workload == "batch_cfg3":
        return run_reference_batch(args)
    X, _, n, reps = inputs.workload(args.workload)
    N = X.shape[0]
    cores = oracle.max_threads()
    pairs = args.ref_pairs
    for w in range(args.warmup):
        cpu_oracle_rate(X, reps, max(256, pairs // 8), 100 + w)
    times = []
    for s in range(args.steps):
        _, dt = cpu_oracle_rate(X, reps, pairs, 1000 + s)
        times.append(dt)
    per_step = sum(times) / len(times)
    value = pairs / per_step
    line = {
        "impl": "reference", "metric": "gram_entries_per_s", "value": value, "unit": "entries/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "n_qubits": n, "reps": reps, "n_points": N,
                   "entries": "unique pairs i<=j", "note": "CPU oracle on a random sample of pairs per step"},
        "cpu_baseline": {"value": value, "unit": "entries/s", "cores": cores, "kind": "oracle",
                         "sample": f"{pairs} random pairs of the {N}-point Gram per step"},
        "e2e": {"value": value, "unit": "entries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_reference_batch(args):
    """CPU oracle on the 32-job batch: per step, a random sample of each job's pairs
    in proportion to its share of the batch's pairs."""
    from oracle import oracle
    spec = inputs.batch_jobs(seed=3)
    sizes = [X.shape[0] * (X.shape[0] + 1) // 2 for X, _ in spec]
    total = sum(sizes)
    rng = np.random.default_rng(5)
    times = []
    for s in range(args.warmup + args.steps):
        t = 0.0
        for (X, n), sz in zip(spec, sizes):
            k = max(1, int(round(args.ref_pairs * sz / total)))
            a, b = rng.integers(0, X.shape[0], k), rng.integers(0, X.shape[0], k)
            t0 = time.perf_counter()
            oracle.mps_pairs(X, X, np.minimum(a, b), np.maximum(a, b), 2)
            t += time.perf_counter() - t0
        if s >= args.warmup:
            times.append(t)
    per_step = sum(times) / len(times)
    value = args.ref_pairs / per_step
    print(json.dumps({
        "impl": "reference", "metric": "gram_entries_per_s", "value": value, "unit": "entries/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "batch_cfg3", "jobs": len(spec), "reps": 2},
        "cpu_baseline": {"value": value, "unit": "entries/s", "cores": oracle.max_threads(), "kind": "oracle",
                         "sample": f"~{args.ref_pairs} pairs per step, drawn from every job by its share"},
        "e2e": {"value": value, "unit": "entries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}), flush=True)
    return 0


def run_ours(args):
    import torch

    from paper_2405_02630_gb300 import build as qbuild
    from paper_2405_02630_gb300 import qsvm

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    qbuild.build()
    qsvm.lib()

    X, Xte, n, reps = inputs.workload(args.workload, scale=world ** 0.5)
    N = X.shape[0]
    Nte = 0 if Xte is None else Xte.shape[0]
    prec = args.precision
    P = qsvm.PRECISIONS[prec]
    Xd = torch.from_numpy(X).to(dev)
    mps = torch.empty(qsvm.qsvm_mps_bytes(n, reps, N, P), dtype=torch.uint8, device=dev)
    K = torch.empty((N, N), dtype=torch.float64, device=dev)
    tb, te = qsvm.qsvm_gram_partition(N, reps, P, world, rank)
    # test x train cross kernel (workloads with a test set): rows split evenly over ranks
    a0, a1 = (Nte * rank) // world, (Nte * (rank + 1)) // world
    if Nte:
        Xted = torch.from_numpy(Xte).to(dev)
        mps_te = torch.empty(qsvm.qsvm_mps_bytes(n, reps, Nte, P), dtype=torch.uint8, device=dev)
        Kx = torch.empty((Nte, N), dtype=torch.float64, device=dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    td = qsvm.qsvm_gram_tile_dim(reps, P)

    def tiles_pairs(lo, hi, pcode=P):
        # pairs contracted by tiles [lo, hi) of the Gram's tile order (tile size depends on the precision)
        tdim = qsvm.qsvm_gram_tile_dim(reps, pcode)
        tot = 0
        for bb in range(lo, hi):
            ti, tj = qsvm.qsvm_gram_tile_coords(N, reps, pcode, bb)
            ni, nj = min(tdim, N - ti * tdim), min(tdim, N - tj * tdim)
            tot += ni * (ni + 1) // 2 if ti == tj else ni * nj
        return tot

    pairs_rank = tiles_pairs(tb, te) + (a1 - a0) * N
    total_pairs = N * (N + 1) // 2 + Nte * N

    # pipeline shape: the autotuner times every shape on a Gram of up to 4096 of the
    # workload's points (untimed setup) and keeps the fastest for the timed steps
    pipeline = {"autotuned": False}
    if args.config is not None:  # a fixed configuration (e.g. the one the autotuner picked, for a profiler run)
        qsvm.qsvm_set_config(reps, P, args.config)
    elif not args.no_autotune:
        Nt = min(N, 4096)
        mps_t = torch.empty(qsvm.qsvm_mps_bytes(n, reps, Nt, P), dtype=torch.uint8, device=dev)
        qsvm.qsvm_build_mps(Xd[:Nt].contiguous(), reps, P, mps=mps_t, stream=stream)
        K_t = torch.empty((Nt, Nt), dtype=torch.float64, device=dev)
        best, tune_ms = qsvm.qsvm_autotune(mps_t, Nt, n, reps, P, K_t, stream=stream)
        torch.cuda.synchronize()
        del mps_t, K_t
        pipeline = {"autotuned": True, "tuned_on_points": Nt, "config": best,
                    "tune_ms": [round(v, 3) for v in tune_ms]}
    cfg = qsvm.qsvm_get_config(reps, P)  # -1: the library's default shape for (reps, precision)
    pipeline["config"] = cfg
    if cfg >= 0:
        pipeline["sites_per_chunk"], pipeline["stages"] = qsvm.qsvm_config_info(cfg, reps, P)
    side, tpp = qsvm.qsvm_config_tile(cfg, reps, P)
    pipeline["cta_pairs"] = f"{side}x{side}"
    pipeline["threads_per_pair"] = tpp
    pipeline["configs_searched"] = qsvm.qsvm_num_configs() if pipeline["autotuned"] else 0

    LK = LKx = None  # ln K outputs, allocated for the timing with ln K written

    def step(prec_code=P, tile_range=(tb, te), with_logk=False):
        qsvm.qsvm_build_mps(Xd, reps, prec_code, mps=mps, stream=stream)
        if Nte:
            qsvm.qsvm_build_mps(Xted, reps, prec_code, mps=mps_te, stream=stream)
        ev_mid = torch.cuda.Event(enable_timing=True)
        ev_mid.record(stream)
        qsvm.qsvm_kernel_gram_tiles(mps, N, n, reps, prec_code, tile_range[0], tile_range[1], K,
                                    logK=LK if with_logk else None, stream=stream)
        if Nte and a1 > a0:
            stride = qsvm.qsvm_mps_point_bytes(n, reps, prec_code)
            qsvm.qsvm_kernel_cross(mps_te[a0 * stride:], a1 - a0, mps, N, n, reps, prec_code, K=Kx[a0:a1],
                                   logK=LKx[a0:a1] if with_logk else None, stream=stream)
        return ev_mid

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        step()
    barrier()

    sampler = ClockSampler(int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0])
                           if os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0].isdigit() else local)
    sampler.start()
    step_ms, kern_ms = [], []
    for _ in range(args.steps):
        flush.fill_(1.0)
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        emid = step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        step_ms.append(e0.elapsed_time(e1))
        kern_ms.append(emid.elapsed_time(e1))
    barrier()
    clocks = sampler.stop()
    status = qsvm.qsvm_device_status()
    if status != 0:
        raise RuntimeError(f"device status {status}")

    # the same step with ln K written beside K (the default output of the Python API):
    # reported beside the K-only headline, same timing rules, up to three steps
    LK = torch.empty((N, N), dtype=torch.float64, device=dev)
    LKx = torch.empty((Nte, N), dtype=torch.float64, device=dev) if Nte else None
    step(with_logk=True)
    barrier()
    log_ms = []
    for _ in range(max(1, min(args.steps, 3))):
        flush.fill_(1.0)
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(with_logk=True)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        log_ms.append(e0.elapsed_time(e1))
    del LK, LKx
    LK = LKx = None

    ms = sum(step_ms) / len(step_ms)
    kms = sum(kern_ms) / len(kern_ms)
    lms = sum(log_ms) / len(log_ms)
    if world > 1:
        t = torch.tensor([ms, kms, lms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms, kms, lms = float(t[0]), float(t[1]), float(t[2])
    value = total_pairs / (ms * 1e-3)

    # ---- roofline of the dominant kernel (the pair contraction) ----
    cm = factorized_cmacs_per_entry(n, reps, prec)
    algo_flops = 8.0 * cm * pairs_rank
    achieved = algo_flops / (kms * 1e-3) / 1e12
    mhz = SM_MAX_MHZ_NOMINAL
    if prec == "fp64":
        peak = 1.25  # nominal GB300 FP64 rate (TFLOP/s)
        bound = "alu"
    else:
        peak = N_SM * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
        bound = "alu"
    fma_frac = (FMA_PER_CMAC[prec] * 2.0 * cm * pairs_rank / (kms * 1e-3) / 1e12) / peak
    roofline = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": measured_traffic(args.workload, prec, cfg) if world == 1 else None,
                "traffic_unit": "bytes per launch (ncu)",
                "kernel_digest": kernel_digest(),
                "kernel": f"pair_tile_kernel<chi={2 ** reps},{prec}>",
                "peak_basis": (f"{N_SM} SMs x {FP32_LANES_PER_SM} FP32 FMA/clk x 2 x {mhz:.0f} MHz"
                               if prec != "fp64" else "nominal FP64 1.25 TFLOP/s"),
                "algorithmic_flops_per_entry": 8 * cm,
                "block_sparse_flops_per_entry": 8 * structured_cmacs_per_entry(n, reps),
                "dense_equiv_flops_per_entry": 8 * dense_cmacs_per_entry(n, reps),
                # the same launch counted in the dense per-entry work (minimal bonds, no
                # factorization): above the peak because the kernel's form needs less work
                "dense_equiv_tflops": 8.0 * dense_cmacs_per_entry(n, reps) * pairs_rank / (kms * 1e-3) / 1e12,
                "fma_pipe_frac": fma_frac}

    line = {
        "metric": "gram_entries_per_s", "value": value, "unit": "entries/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": {"fp32_split": "f32x2-split", "fp32": "f32",
                                                            "fp64": "f64"}[prec],
        "data": "synthetic",
        "config": {"workload": args.workload, "n_qubits": n, "reps": reps, "n_points": N, "n_test": Nte,
                   "points_scaled_by": round(world ** 0.5, 6),
                   "precision": prec,
                   "entries": "unique Gram pairs i<=j incl. diagonal" + (" + test x train" if Nte else ""),
                   "l2": "flushed (512 MB write) between timed steps", "parallelism": f"tiles{world}"},
        "roofline": roofline,
        "pipeline": pipeline,
        "gpu_launches": (4 if Nte else 2) * args.steps,
        "clocks": clocks,
        "pair_kernel_ms": kms,
        "qubit_pair_sites_per_s": value * n,
        "with_logK": {"ms_per_step": lms, "entries_per_s": total_pairs / (lms * 1e-3), "steps": len(log_ms),
                      "note": "same step with ln K written beside K (the API default); value is K only"},
    }

    if rank == 0 and world == 1 and not args.quick:
        # measured library GEMM ceilings (after the timed region): the FP64 run's fraction
        # is taken against the measured DGEMM rate; the FP32 paths keep the peak derived
        # from unit counts and clock, with their fraction of measured SGEMM beside it
        gp = gemm_peaks(dev)
        roofline["measured_gemm_tflops"] = gp
        roofline["measured_gemm_basis"] = "torch.matmul f64 4096^3 / f32 (TF32 off) 8192^3, best of 3"
        if prec == "fp64":
            roofline["peak"] = gp["f64"]
            roofline["frac"] = achieved / gp["f64"]
            roofline["peak_basis"] = "measured DGEMM (torch.matmul float64 4096^3)"
            roofline["frac_of_nominal_fp64"] = achieved / 1.25
        else:
            roofline["frac_of_measured_sgemm"] = achieved / gp["f32"]
        # accuracy of this run against the CPU oracle on sampled pairs
        from oracle import oracle
        rng = np.random.default_rng(7)
        ns = min(256, N)
        di = rng.choice(N, ns, replace=False)
        ia = np.concatenate([di, rng.integers(0, N, ns)])
        ib = np.concatenate([di, rng.integers(0, N, ns)])
        Ko, _ = oracle.mps_pairs(X, X, ia, ib, reps)
        Kg = K[torch.from_numpy(ia).to(dev), torch.from_numpy(ib).to(dev)].cpu().numpy()
        acc = {"pairs": int(ia.size), "max_abs_dK": float(np.max(np.abs(Kg - Ko))),
               "mean_abs_dK": float(np.mean(np.abs(Kg - Ko))),
               "max_abs_diag_minus_1": float(np.max(np.abs(np.diag(K.cpu().numpy()) - 1)))}
        if Nte:
            xa, xb = rng.integers(0, Nte, ns), rng.integers(0, N, ns)
            Kxo, _ = oracle.mps_pairs(Xte, X, xa, xb, reps)
            Kxg = Kx[torch.from_numpy(xa).to(dev), torch.from_numpy(xb).to(dev)].cpu().numpy()
            acc["cross_pairs"] = int(ns)
            acc["cross_max_abs_dK"] = float(np.max(np.abs(Kxg - Kxo)))
        # near-duplicate pairs, K spread over (0, 1): where |dK| is informative.  A Gram
        # of 24 base rows with three perturbed copies each, shuffled, through the same
        # symmetric Gram kernel as the timed step: such pairs fall in diagonal tiles
        # (masked half tile, mirror) and in off-diagonal tiles.  Every entry i < j.
        Xnd, _ = inputs.near_duplicate_clusters(24, 4, n, 40)
        Knd_o, LKnd_o = oracle.mps_gram(Xnd, reps)
        Knd, LKnd = qsvm.gram(torch.from_numpy(Xnd).to(dev), reps, prec, logK=True)
        Knd, LKnd = Knd.cpu().numpy(), LKnd.cpu().numpy()
        iu, ju = np.triu_indices(Xnd.shape[0], 1)
        d = np.abs(Knd[iu, ju] - Knd_o[iu, ju])
        inf = Knd_o[iu, ju] > 0.1
        td_nd = qsvm.qsvm_gram_tile_dim(reps, P)
        big = Knd_o[iu, ju] > 1e-300  # ln K compared where the oracle's K is a normal double
        dlog10 = np.abs(LKnd[iu, ju] - LKnd_o[iu, ju])[big] / np.log(10.0)
        acc["near_dup"] = {"kernel": "qsvm_kernel_gram (symmetric Gram)", "points": int(Xnd.shape[0]),
                           "pairs": int(d.size), "K_range": [float(Knd_o[iu, ju].min()), float(Knd_o[iu, ju].max())],
                           "pairs_K_above_0.1": int(inf.sum()),
                           "of_which_in_diagonal_tiles": int((inf & (iu // td_nd == ju // td_nd)).sum()),
                           "max_abs_dK": float(d.max()), "mean_abs_dK": float(d.mean()),
                           "max_abs_dK_K_above_0.1": float(d[inf].max()),
                           "max_abs_dlog10K": float(dlog10.max()) if dlog10.size else None,
                           "log_pairs": int(dlog10.size)}
        line["accuracy_vs_oracle"] = acc
        # the FP64 path on the same GPU over the whole Gram (speedup report); with
        # --sampled-fp64 only on its first 1/64 of the tiles
        if prec != "fp64":
            nt64 = qsvm.qsvm_gram_num_tiles(N, reps, 0)
            nt = max(1, nt64 // 64) if args.sampled_fp64 else nt64
            mps64 = torch.empty(qsvm.qsvm_mps_bytes(n, reps, N, 0), dtype=torch.uint8, device=dev)
            qsvm.qsvm_build_mps(Xd, reps, "fp64", mps=mps64)
            K64 = torch.full((N, N), float("nan"), dtype=torch.float64, device=dev)
            qsvm.qsvm_kernel_gram_tiles(mps64, N, n, reps, "fp64", 0, nt, K64)  # warm
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            qsvm.qsvm_kernel_gram_tiles(mps64, N, n, reps, "fp64", 0, nt, K64)
            e1.record()
            torch.cuda.synchronize()
            sub_pairs = tiles_pairs(0, nt, 0)
            fp64_rate = sub_pairs / (e0.elapsed_time(e1) * 1e-3)
            m = ~torch.isnan(K64)
            dk = (K[m] - K64[m]).abs()
            line["fp64_same_gpu"] = {"entries_per_s": fp64_rate, "tiles_timed": nt, "tiles_total": nt64,
                                     "speedup_of_" + prec: value / fp64_rate,
                                     "pair_kernel_speedup": (pairs_rank / (kms * 1e-3)) / fp64_rate,
                                     "entries_compared": int(m.sum()),
                                     "max_abs_dK_vs_fp64": float(dk.max()), "mean_abs_dK_vs_fp64": float(dk.mean())}
            if Nte and not args.sampled_fp64:
                mte64 = qsvm.qsvm_build_mps(torch.from_numpy(Xte).to(dev), reps, "fp64")
                Kx64, _ = qsvm.qsvm_kernel_cross(mte64, Nte, mps64, N, n, reps, "fp64")
                dx = (Kx - Kx64).abs()
                line["fp64_same_gpu"]["cross_max_abs_dK_vs_fp64"] = float(dx.max())
                line["fp64_same_gpu"]["cross_mean_abs_dK_vs_fp64"] = float(dx.mean())
                del Kx64, mte64
            del K64, mps64
        # CPU baseline: the oracle on the host cores, bounded sample
        rate, dt = cpu_oracle_rate(X, reps, args.cpu_pairs, 11)
        line["cpu_baseline"] = {"value": rate, "unit": "entries/s", "cores": oracle.max_threads(), "kind": "oracle",
                                "sample": f"{args.cpu_pairs} random pairs of the {N}-point Gram ({dt:.1f} s)"}

    if not args.no_e2e:
        # end to end through the C ABI with host buffers: qsvm_gram_host copies pinned host X
        # to the device, builds, computes the Gram and copies K back to pinned host memory
        # (row bands overlapped with the remaining launches); qsvm_cross_host does the same
        # for the test x train kernel.  A rank of a sharded run (world > 1) computes its
        # tile range on device buffers and copies the whole matrices.
        Xh = torch.from_numpy(X).pin_memory()
        Kh = torch.empty((N, N), dtype=torch.float64).pin_memory()
        Xteh = torch.from_numpy(Xte).pin_memory() if Nte else None
        Kxh = torch.empty((Nte, N), dtype=torch.float64).pin_memory() if Nte else None
        ws_h = torch.empty(qsvm.qsvm_gram_host_workspace_bytes(N, n, reps, P), dtype=torch.uint8, device=dev) \
            if world == 1 else None
        ws_x = torch.empty(qsvm.qsvm_cross_host_workspace_bytes(Nte, N, n, reps, P), dtype=torch.uint8,
                           device=dev) if world == 1 and Nte else None
        e2e_ms = []
        for it in range(max(2, min(args.steps, 3)) + 1):
            flush.fill_(1.0)
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if world == 1:
                qsvm.gram_host(Xh, reps, P, K=Kh, logK=False, ws=ws_h, stream=stream)
                if Nte:
                    qsvm.cross_host(Xteh, Xh, reps, P, K=Kxh, logK=False, ws=ws_x, stream=stream)
            else:
                Xd.copy_(Xh, non_blocking=True)
                if Nte:
                    Xted.copy_(Xteh, non_blocking=True)
                step()
                Kh.copy_(K, non_blocking=True)
                if Nte:
                    Kxh.copy_(Kx, non_blocking=True)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            if it > 0:
                e2e_ms.append(e0.elapsed_time(e1))
        em = sum(e2e_ms) / len(e2e_ms)
        if world > 1:
            t = torch.tensor([em], dtype=torch.float64, device=dev)
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            em = float(t[0])
        line["e2e"] = {"value": total_pairs / (em * 1e-3), "unit": "entries/s",
                       "h2d_bytes_per_step": int(X.nbytes) + (int(Xte.nbytes) if Nte else 0),
                       "d2h_bytes_per_step": int((N + Nte) * N * 8)}

    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_batch(args):
    """32 uneven Gram jobs (n from {16..784}, N in [64, 1024], reps = 2): one persistent
    launch replayed from a CUDA graph, against per-job launches in the same precision
    and per-job FP64 launches.  Single GPU: under torchrun only rank 0 runs."""
    import torch

    from paper_2405_02630_gb300 import build as qbuild
    from paper_2405_02630_gb300 import qsvm

    rank, world, local = dist_env()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    qbuild.build()
    qsvm.lib()
    reps, prec = 2, args.precision
    P = qsvm.PRECISIONS[prec]
    stream = torch.cuda.current_stream(dev)
    spec = inputs.batch_jobs(seed=3)
    Xs = [torch.from_numpy(X).to(dev) for X, _ in spec]

    def make(pcode):
        jobs = []
        for (X, n), Xd in zip(spec, Xs):
            N = X.shape[0]
            jobs.append({"mps": torch.empty(qsvm.qsvm_mps_bytes(n, reps, N, pcode), dtype=torch.uint8, device=dev),
                         "n_points": N, "n_qubits": n, "X": Xd,
                         "K": torch.empty((N, N), dtype=torch.float64, device=dev), "logK": None})
        return jobs

    def build_all(jobs, pcode):
        for j in jobs:
            qsvm.qsvm_build_mps(j["X"], reps, pcode, mps=j["mps"], stream=stream)

    jobs = make(P)
    ws = torch.empty(qsvm.qsvm_batch_workspace_bytes(len(jobs)), dtype=torch.uint8, device=dev)
    total_pairs = sum(j["n_points"] * (j["n_points"] + 1) // 2 for j in jobs)
    algo_flops = sum(8.0 * factorized_cmacs_per_entry(j["n_qubits"], reps, prec) * j["n_points"] * (j["n_points"] + 1) / 2
                     for j in jobs)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    build_all(jobs, P)
    torch.cuda.synchronize()
    plan = qsvm.qsvm_batch_plan_create(jobs, reps, prec, ws)

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        tot, kern = [], []
        for _ in range(steps):
            flush.fill_(1.0)
            torch.cuda.synchronize()
            e0, em, e1 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record(stream)
            fn(em)
            e1.record(stream)
            torch.cuda.synchronize()
            tot.append(e0.elapsed_time(e1))
            kern.append(em.elapsed_time(e1))
        return sum(tot) / len(tot), sum(kern) / len(kern)

    def step_batch(em=None):
        build_all(jobs, P)
        if em is not None:
            em.record(stream)
        plan.launch(stream)

    def step_perjob(em=None):
        build_all(jobs, P)
        if em is not None:
            em.record(stream)
        for j in jobs:
            qsvm.qsvm_kernel_gram(j["mps"], j["n_points"], j["n_qubits"], reps, prec, K=j["K"], stream=stream)

    sampler = ClockSampler(local)
    sampler.start()
    ms, kms = timed(step_batch, args.steps, args.warmup)
    clocks = sampler.stop()
    Kb = [j["K"].clone() for j in jobs]
    ms_pj, kms_pj = timed(step_perjob, max(1, args.steps // 2), 1)
    same = all(torch.equal(a, j["K"]) for a, j in zip(Kb, jobs))
    jobs64 = make(0)

    def step_fp64(em=None):
        build_all(jobs64, 0)
        if em is not None:
            em.record(stream)
        for j in jobs64:
            qsvm.qsvm_kernel_gram(j["mps"], j["n_points"], j["n_qubits"], reps, "fp64", K=j["K"], stream=stream)

    ms64, kms64 = timed(step_fp64, 1, 1)
    dk = max(float((a - j["K"]).abs().max()) for a, j in zip(Kb, jobs64))
    value = total_pairs / (ms * 1e-3)
    peak = N_SM * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ_NOMINAL * 1e6 / 1e12
    achieved = algo_flops / (kms * 1e-3) / 1e12
    line = {
        "metric": "gram_entries_per_s", "value": value, "unit": "entries/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": {"fp32_split": "f32x2-split", "fp32": "f32", "fp64": "f64"}[prec],
        "data": "synthetic",
        "config": {"workload": "batch_cfg3", "jobs": len(jobs), "reps": reps, "precision": prec,
                   "n_qubits": sorted({j["n_qubits"] for j in jobs}),
                   "n_points_range": [min(j["n_points"] for j in jobs), max(j["n_points"] for j in jobs)],
                   "entries": "unique pairs i<=j over all jobs", "launch": "persistent kernel replayed from a CUDA graph",
                   "l2": "flushed (512 MB write) between timed steps"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": None, "kernel": f"pair_persistent_kernel<chi=4,{prec}>"},
        "gpu_launches": (len(jobs) + 1) * args.steps,
        "clocks": clocks,
        "contraction_ms": kms,
        "per_job_launches": {"entries_per_s": total_pairs / (ms_pj * 1e-3), "contraction_ms": kms_pj,
                             "bit_identical_to_batch": same},
        "per_job_fp64": {"entries_per_s": total_pairs / (ms64 * 1e-3), "contraction_ms": kms64,
                         "max_abs_dK_batch_vs_fp64": dk},
    }
    plan.close()
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32_split", choices=["fp32_split", "fp32", "fp64"])
    ap.add_argument("--workload", default="gram_n784_r2_N8192")
    ap.add_argument("--cpu-pairs", type=int, default=65536)
    ap.add_argument("--ref-pairs", type=int, default=16384)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--quick", action="store_true", help="skip the accuracy, FP64 and CPU side measurements")
    ap.add_argument("--sampled-fp64", action="store_true",
                    help="time the FP64 comparison path on the first 1/64 of the Gram's tiles only")
    ap.add_argument("--config", type=int, default=None,
                    help="run this pipeline configuration (qsvm_set_config index) instead of autotuning")
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip the autotuner (by default it picks the pipeline shape and the pairs per CTA on up "
                         "to 4096 of the workload's points before timing)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch_cfg3":
        return run_batch(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
