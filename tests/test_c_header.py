"""include/qsvm.h is a C header: a C99 program compiles against it with all warnings
as errors, links libqsvm.so, and calls the host-only entry points (no GPU needed)."""
import os
import shutil
import subprocess

import pytest

from paper_2405_02630_gb300 import qsvm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include "qsvm.h"

int main(void) {
  int64_t begin = -1, end = -1, total;
  printf("version %s\n", qsvm_version());
  printf("record %zu %zu %zu\n", qsvm_mps_record_bytes(2, QSVM_FP64), qsvm_mps_record_bytes(2, QSVM_FP32),
         qsvm_mps_record_bytes(2, QSVM_FP32_SPLIT));
  printf("mps %zu\n", qsvm_mps_bytes(784, 2, 8192, QSVM_FP32_SPLIT));
  total = qsvm_gram_num_tiles(8192, 2, QSVM_FP32_SPLIT);
  if (qsvm_gram_partition(8192, 2, QSVM_FP32_SPLIT, 4, 3, &begin, &end) != QSVM_OK) return 1;
  printf("tiles %lld %lld %lld %d\n", (long long)total, (long long)begin, (long long)end,
         (int)qsvm_gram_tile_dim(2, QSVM_FP32_SPLIT));
  /* an argument error comes back as a status code with a message, no CUDA call made */
  printf("err %d %s\n", (int)qsvm_kernel_gram(NULL, 16, 8, 2, QSVM_FP64, NULL, 16, NULL, 0, NULL),
         qsvm_last_error() ? "msg" : "none");
  return 0;
}
"""


@pytest.mark.skipif(shutil.which("gcc") is None, reason="no C compiler")
def test_c_program_against_header(tmp_path):
    libdir = os.path.dirname(qsvm.lib()._name)
    src = tmp_path / "abi.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "abi"
    cmd = ["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o",
           str(exe), "-L", libdir, "-lqsvm", f"-Wl,-rpath,{libdir}"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stderr
    lines = dict(line.split(" ", 1) for line in out.stdout.strip().splitlines())
    assert lines["record"] == "32 96 64"
    assert int(lines["mps"]) == 2 * 8192 * 785 * 64
    total, begin, end, tdim = map(int, lines["tiles"].split())
    assert tdim == 16 and total == 512 * 513 // 2 and 0 < begin < end == total
    code, msg = lines["err"].split()
    assert int(code) == qsvm.QSVM_ERR_ARG and msg == "msg"
