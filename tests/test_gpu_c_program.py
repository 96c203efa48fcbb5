"""The C ABI driven from a plain C program on the GPU: cudaMalloc'd buffers, MPS build
and Grams in split FP32 and FP64 through include/qsvm.h, checked for K_ii = 1, exact
symmetry and split-vs-FP64 agreement; then the host-buffer calls qsvm_gram_host
(bit-identical to the device Gram) and qsvm_cross_host (against the FP64 Gram's rows).  No Python or PyTorch on the data path."""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")

PROGRAM = r"""
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <cuda_runtime.h>
#include "qsvm.h"

#define CK(x) do { if ((x) != 0) { fprintf(stderr, "fail %s: %s\n", #x, qsvm_last_error()); return 1; } } while (0)

static int gram(const double* dX, int N, int n, int reps, int prec, double* K) {
  size_t mb = qsvm_mps_bytes(n, reps, N, prec);
  void* mps = NULL;
  double* dK = NULL;
  if (cudaMalloc(&mps, mb) != cudaSuccess || cudaMalloc((void**)&dK, sizeof(double) * N * N) != cudaSuccess) return 1;
  CK(qsvm_build_mps(dX, N, n, reps, prec, mps, mb, NULL));
  CK(qsvm_kernel_gram(mps, N, n, reps, prec, dK, N, NULL, 0, NULL));
  if (cudaMemcpy(K, dK, sizeof(double) * N * N, cudaMemcpyDeviceToHost) != cudaSuccess) return 1;
  cudaFree(mps);
  cudaFree(dK);
  return 0;
}

int main(void) {
  const int N = 37, n = 48, reps = 2;
  double* X = (double*)malloc(sizeof(double) * N * n);
  double *K1 = (double*)malloc(sizeof(double) * N * N), *K2 = (double*)malloc(sizeof(double) * N * N);
  for (int i = 0; i < N * n; ++i) X[i] = 3.14159265358979 * fmod(0.6180339887 * (i + 1), 1.0);
  double* dX = NULL;
  if (cudaMalloc((void**)&dX, sizeof(double) * N * n) != cudaSuccess) return 1;
  cudaMemcpy(dX, X, sizeof(double) * N * n, cudaMemcpyHostToDevice);
  if (gram(dX, N, n, reps, QSVM_FP32_SPLIT, K1) || gram(dX, N, n, reps, QSVM_FP64, K2)) return 1;
  double diag = 0, asym = 0, dk = 0, kmin = 1, kmax = 0;
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) {
      double a = K1[i * N + j];
      if (i == j && fabs(a - 1) > diag) diag = fabs(a - 1);
      if (a != K1[j * N + i]) asym = 1;
      if (fabs(a - K2[i * N + j]) > dk) dk = fabs(a - K2[i * N + j]);
      if (a < kmin) kmin = a;
      if (a > kmax) kmax = a;
    }
  /* host in, host out: the Gram (bit-identical to the device path) and 10 test points x N */
  const int Nt = 10;
  size_t wg = qsvm_gram_host_workspace_bytes(N, n, reps, QSVM_FP32_SPLIT, 0);
  size_t wx = qsvm_cross_host_workspace_bytes(Nt, N, n, reps, QSVM_FP32_SPLIT, 0);
  void *wsg = NULL, *wsx = NULL;
  double *K3 = (double*)malloc(sizeof(double) * N * N), *Kx = (double*)malloc(sizeof(double) * Nt * N);
  if (cudaMalloc(&wsg, wg) != cudaSuccess || cudaMalloc(&wsx, wx) != cudaSuccess) return 1;
  CK(qsvm_gram_host(X, N, n, reps, QSVM_FP32_SPLIT, K3, N, NULL, 0, wsg, wg, NULL));
  CK(qsvm_cross_host(X, Nt, X, N, n, reps, QSVM_FP32_SPLIT, Kx, N, NULL, 0, wsx, wx, NULL));
  if (cudaDeviceSynchronize() != cudaSuccess) return 1;
  double hostdiff = 0, crossdiff = 0;
  for (int i = 0; i < N * N; ++i)
    if (K3[i] != K1[i]) hostdiff = 1;
  for (int i = 0; i < Nt; ++i)
    for (int j = 0; j < N; ++j)
      if (fabs(Kx[i * N + j] - K2[i * N + j]) > crossdiff) crossdiff = fabs(Kx[i * N + j] - K2[i * N + j]);
  int32_t status = -1;
  CK(qsvm_device_status(NULL, 0, &status));
  printf("diag %.3e asym %g dk %.3e kmin %.3e kmax %.6f hostdiff %g crossdk %.3e status %d\n", diag, asym, dk, kmin,
         kmax, hostdiff, crossdiff, (int)status);
  return 0;
}
"""


@pytest.mark.skipif(shutil.which("gcc") is None, reason="no C compiler")
def test_c_program_end_to_end(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_02630_gb300 import qsvm
    qsvm.lib()
    libdir = os.path.dirname(qsvm.LIB_PATH)
    src = tmp_path / "gram.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "gram"
    cmd = ["gcc", "-std=c99", "-O2", "-Wall", "-I", os.path.join(ROOT, "include"), "-I", os.path.join(CUDA, "include"),
           str(src), "-o", str(exe), "-L", libdir, "-lqsvm", f"-Wl,-rpath,{libdir}",
           "-L", os.path.join(CUDA, "lib64"), "-lcudart_static", "-ldl", "-lpthread", "-lrt", "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stdout + out.stderr
    v = out.stdout.split()
    vals = dict(zip(v[0::2], v[1::2]))
    assert float(vals["diag"]) <= 1e-6 and float(vals["asym"]) == 0.0
    assert float(vals["dk"]) <= 1e-6 and 0.0 <= float(vals["kmin"]) and float(vals["kmax"]) <= 1.0 + 1e-6
    assert float(vals["hostdiff"]) == 0.0 and float(vals["crossdk"]) <= 1e-6
    assert int(vals["status"]) == 0
