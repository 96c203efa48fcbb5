"""The GPU state-vector Gram (Algorithm 1's recipe) against the CPU oracle, and
against the GPU MPS path at qubit counts the CPU state vector handles slowly:
two GPU constructions that share no code must agree."""
import numpy as np
import pytest

from paper_2405_02630_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_02630_gb300 import qsvm
    qsvm.lib()
    return qsvm


@pytest.mark.parametrize("n,reps,N", [(1, 2, 5), (2, 1, 9), (5, 3, 17), (8, 2, 16), (10, 2, 33), (7, 4, 12)])
def test_sv_gram_vs_oracle(q, oracle, n, reps, N):
    X = inputs.uniform_features(N, n, 300 + n + reps)
    K = q.qsvm_sv_gram(torch.from_numpy(X).cuda(), reps).cpu().numpy()
    Ko = oracle.sv_gram(X, reps)
    assert np.max(np.abs(K - Ko)) <= 1e-12
    assert np.array_equal(K, K.T)


@pytest.mark.parametrize("n,reps", [(14, 2), (16, 3), (18, 2)])
def test_sv_gram_vs_gpu_mps(q, n, reps):
    N = 40
    X = torch.from_numpy(inputs.mnist_like_features(N, n, 400 + n)).cuda()
    Ksv = q.qsvm_sv_gram(X, reps)
    Kmps, _ = q.gram(X, reps, "fp64")
    assert float((Ksv - Kmps).abs().max()) <= 1e-10
    Ksplit, _ = q.gram(X, reps, "fp32_split")
    assert float((Ksv - Ksplit).abs().max()) <= 1e-6
