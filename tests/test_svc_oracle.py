"""The oracle's SVC (SMO on a precomputed kernel) pinned against scikit-learn's
libsvm solver of the same C-SVC dual and against the KKT conditions of Eq. 1-2's
dual."""
import numpy as np
import pytest


def _kkt_ok(K, y, a, b, C, eps=1e-5):
    f = (a * y) @ K + b
    yf = y * f
    free = (a > 1e-9) & (a < C - 1e-9)
    return (abs(float(a @ y)) < 1e-8 and np.all(np.abs(yf[free] - 1) < eps)
            and np.all(yf[a <= 1e-9] > 1 - eps) and np.all(yf[a >= C - 1e-9] < 1 + eps))


@pytest.mark.parametrize("C", [0.1, 1.0, 10.0])
@pytest.mark.parametrize("kind", ["quantum", "rbf"])
def test_oracle_svc_matches_libsvm(oracle, C, kind):
    sk = pytest.importorskip("sklearn.svm")
    rng = np.random.default_rng(int(C * 10) + len(kind))
    X = rng.random((90, 5)) * np.pi
    y = np.where(np.sin(X[:, 0]) + np.cos(2 * X[:, 1]) > 0.3, 1, -1)
    if kind == "quantum":
        K, _ = oracle.mps_gram(X, 1)
    else:
        d = ((X[:, None, :] - X[None, :, :]) ** 2).sum(-1)
        K = np.exp(-0.5 * d)
    a, b, it = oracle.svc_fit(K, y, C=C, tol=1e-10)
    clf = sk.SVC(kernel="precomputed", C=C, tol=1e-10).fit(K, y)
    assert np.max(np.abs(clf.decision_function(K) - oracle.svc_decision(K, a, y, b))) < 1e-6
    assert _kkt_ok(K, y, a, b, C)
    dual = 0.5 * (a * y) @ K @ (a * y) - a.sum()
    ask = np.zeros(len(y))
    ask[clf.support_] = np.abs(clf.dual_coef_[0])
    dual_sk = 0.5 * (ask * y) @ K @ (ask * y) - ask.sum()
    assert abs(dual - dual_sk) <= 1e-8 * max(1.0, abs(dual_sk))


def test_oracle_svc_index_subset(oracle):
    rng = np.random.default_rng(3)
    X = rng.random((40, 4)) * np.pi
    K, _ = oracle.mps_gram(X, 2)
    idx = np.arange(5, 35)
    y = np.where(X[idx, 0] > np.pi / 2, 1, -1)
    a1, b1, _ = oracle.svc_fit(K, y, C=2.0, tol=1e-10, idx=idx)
    a2, b2, _ = oracle.svc_fit(K[np.ix_(idx, idx)], y, C=2.0, tol=1e-10)
    assert np.array_equal(a1, a2) and b1 == b2
