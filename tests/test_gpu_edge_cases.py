"""Edge cases of the CUDA path: very long chains, degenerate inputs and ragged
shapes, against the oracle or exact values."""
import numpy as np
import pytest

from paper_2405_02630_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32_split": 1e-6}


@pytest.fixture(scope="module")
def q():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_02630_gb300 import qsvm
    qsvm.lib()
    return qsvm


@pytest.mark.parametrize("prec", ["fp64", "fp32_split"])
def test_long_chain_n4096(q, oracle, prec):
    X = inputs.mnist_like_features(12, 4096, 17)
    X[3] = X[0]  # an exact duplicate: K = 1 off the diagonal
    K, LK = q.gram(torch.from_numpy(X).cuda(), 2, prec, logK=True)
    Ko, LKo = oracle.mps_gram(X, 2)
    K = K.cpu().numpy()
    assert np.max(np.abs(K - Ko)) <= TOL[prec]
    assert abs(K[0, 3] - 1.0) <= TOL[prec]
    L = LK.cpu().numpy()
    assert np.all(np.isfinite(L))  # K itself underflows off the diagonal at n = 4096
    assert np.max(np.abs(L - LKo)) <= (1e-8 if prec == "fp64" else 1e-4)


@pytest.mark.parametrize("prec", ["fp64", "fp32_split"])
@pytest.mark.parametrize("reps", [1, 2, 3])
def test_degenerate_inputs(q, oracle, prec, reps):
    n = 50
    X = np.zeros((6, n))          # blank image
    X[1] = np.pi                  # every feature at pi: no ZZ coupling at all
    X[2] = inputs.uniform_features(1, n, 5)[0]
    X[3] = X[2]                   # duplicate
    X[4, ::2] = np.pi             # alternating pattern
    X[5] = 1e-12                  # tiny angles
    K, _ = q.gram(torch.from_numpy(X).cuda(), reps, prec)
    Ko, _ = oracle.mps_gram(X, reps)
    K = K.cpu().numpy()
    assert np.max(np.abs(K - Ko)) <= TOL[prec]
    assert np.max(np.abs(np.diag(K) - 1)) <= TOL[prec]
    assert abs(K[2, 3] - 1) <= TOL[prec] and abs(K[0, 5] - 1) <= 1e-6


@pytest.mark.parametrize("prec", ["fp64", "fp32_split"])
def test_ragged_cross_n784(q, oracle, prec):
    Xtr = inputs.mnist_like_features(37, 784, 8)
    Xte = inputs.mnist_like_features(21, 784, 9)
    Xte[5] = Xtr[7]
    K, _ = q.cross(torch.from_numpy(Xte).cuda(), torch.from_numpy(Xtr).cuda(), 2, prec)
    Ko, _ = oracle.mps_cross(Xte, Xtr, 2)
    K = K.cpu().numpy()
    assert np.max(np.abs(K - Ko)) <= TOL[prec]
    assert abs(K[5, 7] - 1) <= TOL[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32_split"])
def test_long_chain_reps3_n2048(q, oracle, prec):
    """reps = 3 over 2048 sites: K underflows off the diagonal while ln K stays exact."""
    X = inputs.mnist_like_features(6, 2048, 23)
    X[4] = X[1]
    K, LK = q.gram(torch.from_numpy(X).cuda(), 3, prec, logK=True)
    Ko, LKo = oracle.mps_gram(X, 3)
    K, L = K.cpu().numpy(), LK.cpu().numpy()
    assert np.max(np.abs(K - Ko)) <= TOL[prec]
    assert abs(K[1, 4] - 1.0) <= TOL[prec] and np.all(np.isfinite(L))
    assert np.max(np.abs(L - LKo)) <= (1e-8 if prec == "fp64" else 1e-4)


@pytest.mark.parametrize("prec", ["fp64", "fp32_split"])
@pytest.mark.parametrize("reps", [1, 2, 3])
def test_wide_angle_range(q, oracle, prec, reps):
    """Features anywhere in [-3 pi, 3 pi] (the map takes any angle)."""
    X = np.random.default_rng(40 + reps).uniform(-3 * np.pi, 3 * np.pi, (9, 33))
    K, _ = q.gram(torch.from_numpy(X).cuda(), reps, prec)
    Ko, _ = oracle.mps_gram(X, reps)
    assert np.max(np.abs(K.cpu().numpy() - Ko)) <= TOL[prec]
