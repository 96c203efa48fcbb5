#!/usr/bin/env python
"""Benchmark: quantum-kernel Gram entries/s on one GB300 (or N GPUs, strong scaling).

Workload (default): n = 784 qubits (28 x 28 MNIST-like features, 80 % exact zeros,
the rest uniform on (0, 1] * pi; seed 4), reps = 2 (bond dimension 4),
N = 8192 points, the full symmetric 8192 x 8192 Gram.  One step = the whole hot
path: MPS build from the feature matrix (FP64, gate by gate) + the all-pairs
contraction over the upper-triangle tiles (diagonal included) + the mirror
write.  Entries counted = unique pairs contracted, N (N + 1) / 2 per step.

Timing: W untimed warm-up steps, then K steps, each bracketed by CUDA events on
the launching stream with a synchronize on both sides; the L2 (129 MB) is
flushed by writing a 512 MB buffer between timed steps.  Under torchrun each
rank computes a contiguous, pair-balanced share of the tiles of the same Gram
(strong scaling, no collective on the data path); the time is the max over ranks.

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


def dense_cmacs_per_entry(n: int, reps: int) -> int:
    b = [1] + [min(2 ** reps, 2 ** k, 2 ** (n - k)) for k in range(1, n)] + [1]
    return sum(2 * b[k] * b[k + 1] * (b[k] + b[k + 1]) for k in range(n))


# real FP32 FMAs each arithmetic issues per complex MAC of the contraction
FMA_PER_CMAC = {"fp32": 4, "fp32_split": 12, "fp64": 4}


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


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import oracle
    oracle.build()
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
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.workload, "n_qubits": n, "reps": reps, "n_points": N,
                   "entries": "unique pairs i<=j", "note": "CPU oracle on a random sample of pairs per step"},
        "cpu_baseline": {"value": value, "unit": "entries/s", "cores": cores, "kind": "oracle",
                         "sample": f"{pairs} random pairs of the {N}-point Gram per step"},
        "e2e": {"value": value, "unit": "entries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
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

    X, _, n, reps = inputs.workload(args.workload)
    N = X.shape[0]
    prec = args.precision
    P = qsvm.PRECISIONS[prec]
    Xd = torch.from_numpy(X).to(dev)
    mps = torch.empty(qsvm.qsvm_mps_bytes(n, reps, N, P), dtype=torch.uint8, device=dev)
    K = torch.empty((N, N), dtype=torch.float64, device=dev)
    tb, te = qsvm.qsvm_gram_partition(N, reps, P, world, rank)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    td = qsvm.qsvm_gram_tile_dim(reps, P)

    def tiles_pairs(lo, hi):
        # pairs contracted by tiles [lo, hi) of the Gram's tile order
        tot = 0
        for bb in range(lo, hi):
            ti, tj = qsvm.qsvm_gram_tile_coords(N, reps, P, bb)
            ni, nj = min(td, N - ti * td), min(td, N - tj * td)
            tot += ni * (ni + 1) // 2 if ti == tj else ni * nj
        return tot

    pairs_rank = tiles_pairs(tb, te)
    total_pairs = N * (N + 1) // 2

    def step(prec_code=P, tile_range=(tb, te)):
        qsvm.qsvm_build_mps(Xd, reps, prec_code, mps=mps, stream=stream)
        ev_mid = torch.cuda.Event(enable_timing=True)
        ev_mid.record(stream)
        qsvm.qsvm_kernel_gram_tiles(mps, N, n, reps, prec_code, tile_range[0], tile_range[1], K, stream=stream)
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

    ms = sum(step_ms) / len(step_ms)
    kms = sum(kern_ms) / len(kern_ms)
    if world > 1:
        t = torch.tensor([ms, kms], dtype=torch.float64, device=dev)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms, kms = float(t[0]), float(t[1])
    value = total_pairs / (ms * 1e-3)

    # ---- roofline of the dominant kernel (the pair contraction) ----
    cm = structured_cmacs_per_entry(n, reps)
    algo_flops = 8.0 * cm * pairs_rank
    achieved = algo_flops / (kms * 1e-3) / 1e12
    mhz = SM_MAX_MHZ_NOMINAL
    if prec == "fp64":
        peak = 1.25  # nominal GB300 FP64 (recipe table); see the design doc
        bound = "alu"
    else:
        peak = N_SM * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12
        bound = "alu"
    fma_frac = (FMA_PER_CMAC[prec] * 2.0 * cm * pairs_rank / (kms * 1e-3) / 1e12) / peak
    roofline = {"bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": None, "kernel": f"pair_tile_kernel<chi={2 ** reps},{prec}>",
                "peak_basis": (f"{N_SM} SMs x {FP32_LANES_PER_SM} FP32 FMA/clk x 2 x {mhz:.0f} MHz"
                               if prec != "fp64" else "nominal FP64 1.25 TFLOP/s"),
                "algorithmic_flops_per_entry": 8 * cm,
                "dense_equiv_flops_per_entry": 8 * dense_cmacs_per_entry(n, reps),
                "fma_pipe_frac": fma_frac}

    line = {
        "metric": "gram_entries_per_s", "value": value, "unit": "entries/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": {"fp32_split": "f32x2-split", "fp32": "f32",
                                                            "fp64": "f64"}[prec],
        "data": "synthetic",
        "config": {"workload": args.workload, "n_qubits": n, "reps": reps, "n_points": N, "precision": prec,
                   "entries": "unique pairs i<=j incl. diagonal", "l2": "flushed (512 MB write) between timed steps",
                   "parallelism": f"tiles{world}"},
        "roofline": roofline,
        "gpu_launches": 2 * args.steps,
        "clocks": clocks,
        "pair_kernel_ms": kms,
        "qubit_pair_sites_per_s": value * n,
    }

    if rank == 0 and world == 1 and not args.quick:
        # accuracy of this run against the CPU oracle on sampled pairs
        from oracle import oracle
        rng = np.random.default_rng(7)
        di = rng.choice(N, 256, replace=False)
        ia = np.concatenate([di, rng.integers(0, N, 256)])
        ib = np.concatenate([di, rng.integers(0, N, 256)])
        Ko, _ = oracle.mps_pairs(X, X, ia, ib, reps)
        Kg = K[torch.from_numpy(ia).to(dev), torch.from_numpy(ib).to(dev)].cpu().numpy()
        line["accuracy_vs_oracle"] = {"pairs": int(ia.size), "max_abs_dK": float(np.max(np.abs(Kg - Ko))),
                                      "max_abs_diag_minus_1": float(np.max(np.abs(np.diag(K.cpu().numpy()) - 1)))}
        # the FP64 path on the same GPU, on the first tiles of the same Gram (speedup report)
        if prec != "fp64":
            nt = max(1, (te - tb) // 64)
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
            sub_pairs = tiles_pairs(0, nt)
            fp64_rate = sub_pairs / (e0.elapsed_time(e1) * 1e-3)
            m = ~torch.isnan(K64)
            line["fp64_same_gpu"] = {"entries_per_s": fp64_rate, "tiles_timed": nt,
                                     "speedup_of_" + prec: value / fp64_rate,
                                     "pair_kernel_speedup": (pairs_rank / (kms * 1e-3)) / fp64_rate,
                                     "max_abs_dK_vs_fp64": float((K[m] - K64[m]).abs().max())}
            del K64, mps64
        # CPU baseline: the oracle on the host cores, bounded sample
        rate, dt = cpu_oracle_rate(X, reps, args.cpu_pairs, 11)
        line["cpu_baseline"] = {"value": rate, "unit": "entries/s", "cores": oracle.max_threads(), "kind": "oracle",
                                "sample": f"{args.cpu_pairs} random pairs of the {N}-point Gram ({dt:.1f} s)"}

    if not args.no_e2e:
        # end to end through the public API: pinned host X -> device, build, Gram, K -> pinned host
        Xh = torch.from_numpy(X).pin_memory()
        Kh = torch.empty((N, N), dtype=torch.float64).pin_memory()
        e2e_ms = []
        for it in range(max(2, min(args.steps, 3)) + 1):
            flush.fill_(1.0)
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            Xd.copy_(Xh, non_blocking=True)
            step()
            Kh.copy_(K, non_blocking=True)
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
                       "h2d_bytes_per_step": int(X.nbytes), "d2h_bytes_per_step": int(N * N * 8)}

    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
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
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
