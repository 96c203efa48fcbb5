"""Edge cases of the CUDA path: very long chains, degenerate inputs, ragged shapes and
offsets past 32 bits, against the oracle or exact values."""
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


@pytest.mark.parametrize("quarter", [False, True])
def test_gram_offsets_beyond_32_bits(q, oracle, quarter):
    """A 66 000-point Gram (n = 3, split FP32, a ragged last tile): K holds 4.36e9 entries,
    so its element offsets pass 2^32.  Sampled entries, many in the last rows, against the
    oracle, and their mirrors bit-exact; with whole tiles per CTA and with quarter tiles
    (a grid of 34 M CTAs)."""
    N, n, reps = 66000, 3, 2
    X = inputs.uniform_features(N, n, 123)
    if quarter:
        q.qsvm_set_config(reps, "fp32_split", q.qsvm_num_configs() // 2 + 3)
    try:
        K, _ = q.gram(torch.from_numpy(X).cuda(), reps, "fp32_split", logK=False)  # K alone is 35 GB
    finally:
        q.qsvm_set_config(reps, "fp32_split", -1)
    torch.cuda.synchronize()
    assert q.qsvm_device_status() == 0
    rng = np.random.default_rng(5)
    ia = np.concatenate([rng.integers(0, N, 128), rng.integers(65100, N, 128), np.arange(N - 16, N)])
    ib = np.concatenate([rng.integers(0, N, 128), rng.integers(0, N, 128), np.arange(N - 16, N)])
    assert (ia.astype(np.int64) * N + ib).max() >= 2 ** 32
    ta, tb = torch.from_numpy(ia).cuda(), torch.from_numpy(ib).cuda()
    Kg, Kt = K[ta, tb].cpu().numpy(), K[tb, ta].cpu().numpy()
    del K
    torch.cuda.empty_cache()
    Ko, _ = oracle.mps_pairs(X, X, ia, ib, reps)
    assert np.max(np.abs(Kg - Ko)) <= TOL["fp32_split"]
    assert np.array_equal(Kg, Kt)


@pytest.mark.parametrize("prec", ["fp64", "fp32_split"])
def test_cross_record_offsets_beyond_31_bits(q, oracle, prec):
    """8 test points against 70 000 train points at n = 784: the train records span 3.5 GB
    (FP64) or 7 GB (split, two arrays), so record offsets pass 2^31; sampled entries, many
    against the last train points, against the oracle."""
    Ntr, n, reps = 70000, 784, 2
    Xtr = inputs.mnist_like_features(Ntr, n, 124)
    Xte = inputs.mnist_like_features(8, n, 125)
    Xte[3] = Xtr[Ntr - 1]  # K = 1 against the last train point
    K, LK = q.cross(torch.from_numpy(Xte).cuda(), torch.from_numpy(Xtr).cuda(), reps, prec, logK=True)
    torch.cuda.synchronize()
    assert q.qsvm_device_status() == 0
    rng = np.random.default_rng(6)
    ia = np.concatenate([rng.integers(0, 8, 96), rng.integers(0, 8, 96), [3]])
    ib = np.concatenate([rng.integers(0, Ntr, 96), rng.integers(60000, Ntr, 96), [Ntr - 1]])
    ta, tb = torch.from_numpy(ia).cuda(), torch.from_numpy(ib).cuda()
    Kg, Lg = K[ta, tb].cpu().numpy(), LK[ta, tb].cpu().numpy()
    del K, LK
    torch.cuda.empty_cache()
    Ko, LKo = oracle.mps_pairs(Xte, Xtr, ia, ib, reps)
    assert np.max(np.abs(Kg - Ko)) <= TOL[prec]
    assert abs(Kg[-1] - 1.0) <= TOL[prec]
    m = Ko > 1e-300
    assert np.max(np.abs(Lg[m] - LKo[m])) <= (1e-8 if prec == "fp64" else 1e-5)
