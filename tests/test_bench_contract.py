"""bench.py prints one JSON line with the keys its consumers read: the reference arm
(the CPU oracle, no GPU needed) and the GPU arm on a small workload."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
BASE_KEYS = {"metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
             "vs_baseline", "dtype", "data", "config", "e2e", "cpu_baseline"}


def _run(args, timeout):
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT, capture_output=True,
                         text=True, timeout=timeout)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout[-2000:]
    return json.loads(lines[0])


def test_reference_arm_line():
    d = _run(["--impl", "reference", "--workload", "cfg1_n64_r2_N512x256", "--steps", "2", "--warmup", "1",
              "--ref-pairs", "2048"], timeout=600)
    assert BASE_KEYS <= set(d)
    assert d["impl"] == "reference" and d["metric"] == "gram_entries_per_s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]


def test_reference_arm_under_torchrun():
    """Launched like the multi-GPU runs (two ranks): rank 0 alone prints the line, every
    rank exits 0."""
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2", "--master-addr",
           "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus",
           "2", "--workload", "cfg1_n64_r2_N512x256", "--steps", "1", "--warmup", "1", "--ref-pairs", "1024"]
    out = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, out.stdout[-2000:]
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0


def test_traffic_figure_follows_the_kernel_sources(monkeypatch):
    """roofline.traffic is reported only while the pair-kernel sources are the ones its
    ncu capture was taken on."""
    sys.path.insert(0, ROOT)
    import bench
    key = ("gram_n784_r2_N8192", "fp32_split", 9)
    digest, nbytes = bench.MEASURED_TRAFFIC_BYTES[key]
    monkeypatch.setattr(bench, "kernel_digest", lambda: digest)
    assert bench.measured_traffic(*key) == nbytes
    assert bench.measured_traffic("gram_n784_r2_N8192", "fp32_split", 3) is None  # another configuration
    assert bench.measured_traffic("cfg1_n64_r2_N512x256", "fp32_split", 9) is None
    monkeypatch.setattr(bench, "kernel_digest", lambda: "0" * 16)
    assert bench.measured_traffic(*key) is None


@pytest.mark.gpu
def test_gpu_arm_line():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    d = _run(["--workload", "gram_n784_r2_N1024", "--steps", "3", "--warmup", "3"], timeout=900)
    assert BASE_KEYS <= set(d) and "impl" not in d
    assert d["value"] > 0 and d["higher_is_better"] is True and d["gpu_launches"] == 6
    r = d["roofline"]
    assert {"bound", "achieved", "peak", "unit", "frac", "traffic"} <= set(r)
    assert abs(r["frac"] - r["achieved"] / r["peak"]) < 1e-9 and 0 < r["frac"] < 1
    assert d["e2e"]["h2d_bytes_per_step"] > 0 and d["e2e"]["d2h_bytes_per_step"] > 0
    assert {"sm_mhz", "sm_max_mhz", "reasons"} <= set(d["clocks"])
    acc = d["accuracy_vs_oracle"]
    assert acc["max_abs_dK"] <= 1e-6 and acc["near_dup"]["max_abs_dK"] <= 1e-6
    assert acc["near_dup"]["kernel"].startswith("qsvm_kernel_gram") and acc["near_dup"]["pairs_K_above_0.1"] > 0
    p = d["pipeline"]
    assert p["autotuned"] is True and p["configs_searched"] > 12 and "cta_pairs" in p
    f64 = d["fp64_same_gpu"]
    assert f64["tiles_timed"] == f64["tiles_total"] and f64["max_abs_dK_vs_fp64"] <= 1e-6
    assert d["with_logK"]["entries_per_s"] > 0
