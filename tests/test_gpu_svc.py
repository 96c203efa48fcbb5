"""The GPU SVC (one CTA per binary problem) against the oracle's SMO on the same
kernel, and one-vs-one multiclass prediction on synthetic labelled data."""
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


@pytest.mark.parametrize("C", [0.5, 5.0])
def test_gpu_svc_matches_oracle(q, oracle, C):
    rng = np.random.default_rng(int(C * 10))
    X = rng.random((120, 6)) * np.pi
    y = np.where(np.sin(X[:, 0]) * np.cos(X[:, 2]) > 0, 1, -1).astype(np.int8)
    Kd, _ = q.gram(torch.from_numpy(X).cuda(), 2, "fp64")
    K = Kd.cpu().numpy()
    a_o, b_o, _ = oracle.svc_fit(K, y, C=C, tol=1e-9)
    prob = {"idx": torch.arange(120, dtype=torch.int64, device="cuda"), "y": torch.from_numpy(y).cuda(),
            "alpha": torch.empty(120, dtype=torch.float64, device="cuda")}
    b, it = q.qsvm_svc_fit(Kd, [prob], C=C, tol=1e-9)
    F = q.qsvm_svc_decision(Kd, [prob], b).cpu().numpy()[:, 0]
    f_o = oracle.svc_decision(K, a_o, y, b_o)
    assert int(it[0]) > 0
    assert np.max(np.abs(F - f_o)) < 1e-5
    a = prob["alpha"].cpu().numpy()
    assert abs(float(a @ y)) < 1e-8 and a.min() >= 0 and a.max() <= C


def test_gpu_one_vs_one_multiclass(q, oracle):
    from paper_2405_02630_gb300.svc import OneVsOneSVC
    rng = np.random.default_rng(7)
    n, per = 6, 40
    centers = rng.random((4, n)) * np.pi
    Xtr = np.concatenate([np.clip(c + 0.15 * rng.standard_normal((per, n)), 0, np.pi) for c in centers])
    ytr = np.repeat(np.arange(4), per)
    Xte = np.concatenate([np.clip(c + 0.15 * rng.standard_normal((10, n)), 0, np.pi) for c in centers])
    yte = np.repeat(np.arange(4), 10)
    Xd, Xted = torch.from_numpy(Xtr).cuda(), torch.from_numpy(Xte).cuda()
    K, _ = q.gram(Xd, 1, "fp64")
    Kx, _ = q.cross(Xted, Xd, 1, "fp64")
    clf = OneVsOneSVC(C=10.0, tol=1e-9).fit(K, torch.from_numpy(ytr).cuda())
    assert len(clf.pairs) == 6
    pred = clf.predict(Kx).cpu().numpy()
    # the same one-vs-one vote with the oracle's SMO on the same kernels
    Kh, Kxh = K.cpu().numpy(), Kx.cpu().numpy()
    votes = np.zeros((len(yte), 4), dtype=int)
    for a in range(4):
        for b in range(a + 1, 4):
            idx = np.nonzero((ytr == a) | (ytr == b))[0]
            yy = np.where(ytr[idx] == a, 1, -1)
            al, bb, _ = oracle.svc_fit(Kh, yy, C=10.0, tol=1e-9, idx=idx)
            f = oracle.svc_decision(Kxh, al, yy, bb, idx=idx)
            votes[f > 0, a] += 1
            votes[f <= 0, b] += 1
    assert np.array_equal(pred, np.argmax(votes, axis=1))
    assert (pred == yte).mean() >= 0.8
