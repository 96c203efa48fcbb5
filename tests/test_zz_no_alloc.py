"""qsvm_kernel_batch_noalloc: the batch launch for callers that cannot allocate
device memory (serving loops that must not synchronise the device through
cudaMalloc, hosts whose framework allocator owns all device memory).

Its scratch is a fixed array inside the library, reused by every call, so the
test makes two calls in a row with different job sets through the C ABI.  Each
call runs the same persistent kernel on the same records as the workspace entry
point qsvm_kernel_batch, so K and ln K must be bit-identical to it (a stale or
partly rewritten job table would show); each job's K is also checked against the
CPU oracle element by element.  This file is collected last and needs nothing from
the other test files.
"""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-6  # split-FP32 tolerance of the parity tests
LOG_TOL = 1e-5


def _make_jobs(qsvm, specs, reps, prec, seed):
    rng = np.random.default_rng(seed)
    jobs = []
    for N, n in specs:
        Xh = rng.random((N, n)) * np.pi
        mps = qsvm.qsvm_build_mps(torch.from_numpy(Xh).cuda(), reps, prec)
        K = torch.full((N, N), float("nan"), dtype=torch.float64, device="cuda")
        L = torch.full((N, N), float("nan"), dtype=torch.float64, device="cuda")
        jobs.append({"mps": mps, "n_points": N, "n_qubits": n, "K": K, "logK": L, "X": Xh})
    return jobs


def _reference(qsvm, jobs, reps, prec):
    ref = [{**j, "K": torch.empty_like(j["K"]), "logK": torch.empty_like(j["logK"])} for j in jobs]
    ws = torch.empty(qsvm.qsvm_batch_workspace_bytes(len(ref)), dtype=torch.uint8, device="cuda")
    qsvm.qsvm_kernel_batch(ref, reps, prec, ws)
    torch.cuda.synchronize()
    return ref


def test_noalloc_batch_matches_workspace_batch_twice(oracle):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_02630_gb300 import qsvm
    lib = qsvm.lib()
    reps, prec = 2, qsvm.QSVM_FP32_SPLIT
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    job_sets = [[(37, 16), (80, 64), (17, 130), (5, 64)], [(64, 30), (9, 200), (50, 12)]]
    for call, specs in enumerate(job_sets):
        jobs = _make_jobs(qsvm, specs, reps, prec, 10 + call)
        ref = _reference(qsvm, jobs, reps, prec)
        arr = qsvm._jobs_array(jobs)
        rc = lib.qsvm_kernel_batch_noalloc(arr, len(jobs), reps, prec, stream)
        assert rc == qsvm.QSVM_OK, lib.qsvm_last_error().decode()
        torch.cuda.synchronize()
        for j, r in zip(jobs, ref):
            assert not torch.isnan(j["K"]).any() and not torch.isnan(j["logK"]).any()
            assert torch.equal(j["K"], r["K"])
            assert torch.equal(j["logK"], r["logK"])  # -inf where K underflows, on both sides
            Ko, LKo = oracle.mps_gram(j["X"], reps)
            Kg, LKg = j["K"].cpu().numpy(), j["logK"].cpu().numpy()
            assert np.max(np.abs(Kg - Ko)) <= TOL
            m = Ko > 1e-300
            assert np.max(np.abs(LKg[m] - LKo[m])) <= LOG_TOL
    assert qsvm.qsvm_device_status() == 0


def test_noalloc_batch_rejects_too_many_jobs():
    from paper_2405_02630_gb300 import qsvm
    lib = qsvm.lib()
    arr = (qsvm.QsvmJob * 1025)()
    rc = lib.qsvm_kernel_batch_noalloc(arr, 1025, 2, qsvm.QSVM_FP32_SPLIT, None)
    assert rc == qsvm.QSVM_ERR_WORKSPACE
    assert "1024" in lib.qsvm_last_error().decode()
