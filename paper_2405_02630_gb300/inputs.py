"""Seeded synthetic inputs shared by the tests, the bench and the oracle checks.

This module holds no arithmetic of the method: it only draws feature matrices.
The MNIST and Fashion-MNIST sets the paper uses (Sec. 4.2, Sec. 5) are not
available here, so MNIST-like matrices stand in for them: 784 = 28 x 28 features
per point, each feature exactly zero with probability 0.8 (blank pixels), the
rest uniform on (0, 1] and scaled by pi.  Dense workloads draw features iid
uniform on [0, pi).  Everything uses numpy's PCG64 ``default_rng(seed)`` in
float64, row-major (points x features).
"""
from __future__ import annotations

import numpy as np

PI = np.pi

# name -> (n_qubits, reps, n_train, n_test, kind, seed)
WORKLOADS = {
    "cfg0_n8_r2_N16": (8, 2, 16, 0, "uniform", 0),
    "cfg1_n64_r2_N512x256": (64, 2, 512, 256, "uniform", 1),
    "cfg2_n784_r2_N2048x1024": (784, 2, 2048, 1024, "mnist_like", 2),
    "cfg4_n784_r3_N8192": (784, 3, 8192, 0, "mnist_like", 4),
    "gram_n784_r2_N8192": (784, 2, 8192, 0, "mnist_like", 4),
    # smaller cases of the same distribution, for profiler captures
    "gram_n784_r2_N1024": (784, 2, 1024, 0, "mnist_like", 4),
    "gram_n784_r3_N1024": (784, 3, 1024, 0, "mnist_like", 4),
}


def uniform_features(n_points: int, n_features: int, seed: int) -> np.ndarray:
    """iid uniform on [0, pi)."""
    rng = np.random.default_rng(seed)
    return rng.random((n_points, n_features)) * PI


def mnist_like_features(n_points: int, n_features: int, seed: int, p_zero: float = 0.8) -> np.ndarray:
    """Each feature is 0 with probability p_zero, else uniform on (0, 1] times pi."""
    rng = np.random.default_rng(seed)
    zero = rng.random((n_points, n_features)) < p_zero
    val = (1.0 - rng.random((n_points, n_features))) * PI
    return np.where(zero, 0.0, val)


def workload(name: str, scale: float = 1.0):
    """Returns (X_train, X_test or None, n_qubits, reps) for a named workload.  ``scale``
    multiplies the numbers of points (same distribution and seed), e.g. by sqrt(G) to
    keep the pairs per GPU fixed when a Gram is shared by G GPUs."""
    n, reps, ntr, nte, kind, seed = WORKLOADS[name]
    if scale != 1.0:
        ntr, nte = int(round(ntr * scale)), int(round(nte * scale))
    gen = uniform_features if kind == "uniform" else mnist_like_features
    X = gen(ntr + nte, n, seed)
    return X[:ntr], (X[ntr:] if nte else None), n, reps


def near_duplicates(base: np.ndarray, seed: int, frac: float = 0.05,
                    scales=(3e-4, 1e-3, 3e-3, 1e-2, 3e-2, 1e-1)) -> np.ndarray:
    """One perturbed copy per row of ``base``: a random ``frac`` of its features
    move by N(0, scale^2), the scale cycling through ``scales`` row by row, so the
    kernel values between a row and its copy spread over (0, 1)."""
    rng = np.random.default_rng(seed)
    out = base.copy()
    N, n = base.shape
    m = max(1, int(round(frac * n)))
    for r in range(N):
        idx = rng.choice(n, m, replace=False)
        out[r, idx] += scales[r % len(scales)] * rng.standard_normal(m)
    return out


def batch_jobs(seed: int = 3, n_jobs: int = 32, qubits=(16, 64, 128, 256, 512, 784), n_min: int = 64,
               n_max: int = 1024):
    """Uneven Gram jobs: n drawn from ``qubits``, N uniform on [n_min, n_max],
    features uniform on [0, pi).  Returns a list of (X, n_qubits)."""
    rng = np.random.default_rng(seed)
    jobs = []
    for _ in range(n_jobs):
        n = int(rng.choice(qubits))
        N = int(rng.integers(n_min, n_max + 1))
        jobs.append((rng.random((N, n)) * PI, n))
    return jobs


def near_duplicate_clusters(n_base: int, copies: int, n_features: int, seed: int,
                            frac: float = 0.05) -> tuple[np.ndarray, np.ndarray]:
    """A Gram input rich in near-duplicate pairs: ``n_base`` MNIST-like rows, each with
    ``copies`` - 1 perturbed copies (``near_duplicates`` with a different seed per copy),
    all rows shuffled by a seeded permutation so that the copies of one base row land
    both inside one tile of the Gram and in different tiles.  Returns (X, cluster) with
    cluster[r] the base row that row r of X derives from."""
    base = mnist_like_features(n_base, n_features, seed)
    rows = [base] + [near_duplicates(base, seed + 1 + c, frac) for c in range(copies - 1)]
    X = np.concatenate(rows, axis=0)
    cluster = np.tile(np.arange(n_base), copies)
    perm = np.random.default_rng(seed + 1000).permutation(X.shape[0])
    return np.ascontiguousarray(X[perm]), cluster[perm]
