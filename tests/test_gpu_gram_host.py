"""qsvm_gram_host (host X in, host K out, the Gram in chunks of tile bands with the
row bands of K copied out while later chunks compute) against the device path:
bit-identical results for one chunk (small problems) and up to eight, with a
strided host K and with logK; qsvm_cross_host (the test x train kernel of host data, in
row chunks copied out as they finish) against qsvm_build_mps + qsvm_kernel_cross."""
import numpy as np
import pytest
import torch

from paper_2405_02630_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_02630_gb300 import qsvm
    qsvm.lib()
    return qsvm


@pytest.mark.parametrize("prec", ["fp64", "fp32_split", "fp32"])
@pytest.mark.parametrize("N,n,reps", [(1, 2, 2), (37, 13, 1), (300, 24, 2), (2048, 6, 2), (200, 9, 3)])
def test_gram_host_matches_device(q, prec, N, n, reps):
    X = inputs.uniform_features(N, n, 900 + N)
    Kd, Ld = q.gram(torch.from_numpy(X).cuda(), reps, prec, logK=True)
    Xh = torch.from_numpy(X).pin_memory()
    big = torch.full((N, N + 5), -3.0, dtype=torch.float64).pin_memory()
    K, L = q.gram_host(Xh, reps, prec, K=big[:, 2:N + 2], logK=True)
    torch.cuda.synchronize()
    assert q.qsvm_device_status() == 0
    assert torch.equal(K, Kd.cpu()) and torch.equal(L, Ld.cpu())
    B = big.numpy()
    assert np.all(B[:, :2] == -3.0) and np.all(B[:, N + 2:] == -3.0)


def test_gram_host_pageable_and_default_buffers(q):
    """Pageable X, library-allocated pinned K and ln K (the default): same bits as the
    device path; logK=False returns no ln K."""
    N, n = 150, 20
    X = inputs.mnist_like_features(N, n, 77)
    Kd, Ld = q.gram(torch.from_numpy(X).cuda(), 2, "fp32_split")
    K, L = q.gram_host(torch.from_numpy(X), 2, "fp32_split")
    K2, L2 = q.gram_host(torch.from_numpy(X), 2, "fp32_split", logK=False)
    torch.cuda.synchronize()
    assert torch.equal(K, Kd.cpu()) and torch.equal(L, Ld.cpu())
    assert L2 is None and torch.equal(K2, Kd.cpu())


@pytest.mark.parametrize("prec", ["fp64", "fp32_split", "fp32"])
@pytest.mark.parametrize("Na,Nb,n,reps", [(1, 1, 2, 2), (37, 5, 13, 1), (300, 170, 24, 2), (1000, 40, 6, 2),
                                          (129, 200, 9, 3), (2500, 1000, 4, 2)])
def test_cross_host_matches_device(q, prec, Na, Nb, n, reps):
    Xa = inputs.uniform_features(Na, n, 1900 + Na)
    Xb = inputs.uniform_features(Nb, n, 2900 + Nb)
    Kd, Ld = q.cross(torch.from_numpy(Xa).cuda(), torch.from_numpy(Xb).cuda(), reps, prec, logK=True)
    big = torch.full((Na, Nb + 3), -3.0, dtype=torch.float64).pin_memory()
    K, L = q.cross_host(torch.from_numpy(Xa).pin_memory(), torch.from_numpy(Xb), reps, prec, K=big[:, 1:Nb + 1],
                        logK=True)
    torch.cuda.synchronize()
    assert q.qsvm_device_status() == 0
    assert torch.equal(K, Kd.cpu()) and torch.equal(L, Ld.cpu())
    B = big.numpy()
    assert np.all(B[:, :1] == -3.0) and np.all(B[:, Nb + 1:] == -3.0)
