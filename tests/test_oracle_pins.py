"""Pins for the CPU oracle, checked against facts that do not come from the oracle.

Each pin cites what fixes it: the definition K = |<psi_j|psi_i>|^2 (Sec. 2, Eq. 3-4),
the linear-chain feature map of Sec. 3.2, the symmetrisation K + K^T + I of
Algorithms 1-3 (which implies K_ij = K_ji and K_ii = 1), and textbook facts
(a Gram matrix of unit vectors is PSD with entries in [0, 1]; product states
give product kernels; a chain with bond 2^reps has Schmidt rank <= 2^reps).
"""
import itertools

import numpy as np
import pytest

PI = np.pi


def _rand(rng, n, k=1):
    return rng.random((k, n)) * PI


# ---- O1 vs O2: two unrelated constructions of the same circuit (Eq. 4) -----
@pytest.mark.parametrize("n", [1, 2, 3, 4, 6, 9, 12])
@pytest.mark.parametrize("reps", [1, 2, 3])
def test_statevector_matches_mps(oracle, n, reps):
    rng = np.random.default_rng(10 * n + reps)
    X = _rand(rng, n, 4)
    Xs = np.vstack([X, X[:1]])  # includes an identical pair
    for a, b in itertools.combinations_with_replacement(range(len(Xs)), 2):
        k_sv, _ = oracle.sv_kernel_pair(Xs[a], Xs[b], reps)
        k_mps = oracle.mps_overlap(oracle.mps_closed_form(Xs[a], reps), oracle.mps_closed_form(Xs[b], reps), reps)[0]
        assert abs(k_sv - k_mps) <= 1e-12, (a, b, k_sv, k_mps)


# ---- reps = 1: amplitude is a classical Ising sum, summed by brute force ----
def _ising_energy(x, s):
    # f(s) = sum_k x_k z_k + sum_k (pi - x_k)(pi - x_{k+1}) z_k z_{k+1}, z = 1 - 2 s
    z = 1.0 - 2.0 * s
    return z @ x + ((PI - x[:-1]) * (PI - x[1:]) * z[:, :-1] * z[:, 1:]).sum(axis=1)


@pytest.mark.parametrize("n", [2, 5, 10, 13])
def test_reps1_brute_force_ising(oracle, n):
    # After H^n and the diagonal layer, psi_x(s) = 2^{-n/2} exp(-i f_x(s)), so
    # <psi_j|psi_i> = 2^{-n} sum_s exp(-i (f_i(s) - f_j(s))).
    rng = np.random.default_rng(n)
    xi, xj = _rand(rng, n, 2)
    S = ((np.arange(2 ** n)[:, None] >> np.arange(n)[None, :]) & 1).astype(float)
    amp = np.exp(-1j * (_ising_energy(xi, S) - _ising_energy(xj, S))).sum() / 2 ** n
    k_ref = abs(amp) ** 2
    k_sv, _ = oracle.sv_kernel_pair(xi, xj, 1)
    K_mps, _ = oracle.mps_cross(xi[None], xj[None], 1)
    assert abs(k_sv - k_ref) <= 1e-12
    assert abs(K_mps[0, 0] - k_ref) <= 1e-12


# ---- reps = 2: brute-force two-layer path sum ------------------------------
def _reps2_state(x):
    # psi(s2) = 2^{-n} sum_{s1} exp(-i f(s1)) (-1)^{s1.s2} exp(-i f(s2)): H, diagonal
    # layer, H, diagonal layer applied to |0^n>, written as a sum over s1.
    n = x.shape[0]
    S = ((np.arange(2 ** n)[:, None] >> np.arange(n)[None, :]) & 1).astype(float)
    ph = np.exp(-1j * _ising_energy(x, S))
    had = (-1.0) ** (S @ S.T)
    return (had @ ph) * ph / 2 ** n


@pytest.mark.parametrize("n", [2, 4, 7, 9])
def test_reps2_brute_force_path_sum(oracle, n):
    rng = np.random.default_rng(100 + n)
    xi, xj = _rand(rng, n, 2)
    k_ref = abs(np.vdot(_reps2_state(xj), _reps2_state(xi))) ** 2
    k_sv, _ = oracle.sv_kernel_pair(xi, xj, 2)
    K_mps, _ = oracle.mps_cross(xi[None], xj[None], 2)
    assert abs(np.linalg.norm(_reps2_state(xi)) - 1) <= 1e-12
    assert abs(k_sv - k_ref) <= 1e-12 and abs(K_mps[0, 0] - k_ref) <= 1e-12


# ---- no entangler: product state, product kernel -------------------------
def _single_qubit_state(x, reps, phase_gate=False):
    H = np.array([[1, 1], [1, -1]]) / np.sqrt(2)
    if phase_gate:
        Z = np.diag([1.0, np.exp(2j * x)])
    else:
        Z = np.diag([np.exp(-1j * x), np.exp(1j * x)])
    v = np.array([1.0, 0.0], complex)
    for _ in range(reps):
        v = Z @ (H @ v)
    return v


@pytest.mark.parametrize("reps", [1, 2, 3])
def test_no_entangler_product_form(oracle, reps):
    rng = np.random.default_rng(77 + reps)
    n = 7
    xi, xj = _rand(rng, n, 2)
    ref = np.prod([abs(np.vdot(_single_qubit_state(b, reps), _single_qubit_state(a, reps))) ** 2
                   for a, b in zip(xi, xj)])
    k_sv, _ = oracle.sv_kernel_pair(xi, xj, reps, oracle.NO_ENTANGLER)
    K_mps, _ = oracle.mps_cross(xi[None], xj[None], reps, oracle.NO_ENTANGLER)
    assert abs(k_sv - ref) <= 1e-12
    assert abs(K_mps[0, 0] - ref) <= 1e-12
    if reps == 1:  # |<+|RZ(2(x_i - x_j))|+>|^2 = cos^2(x_i - x_j) per qubit
        assert abs(ref - np.prod(np.cos(xi - xj) ** 2)) <= 1e-12
    if reps == 2:  # closed form of the two-layer single-qubit overlap
        f = lambda x, y: (np.cos(x) ** 2 * np.cos(y) ** 2 + np.sin(x) ** 2 * np.sin(y) ** 2
                          + 2 * np.cos(x) * np.cos(y) * np.sin(x) * np.sin(y) * np.cos(2 * (y - x)))
        assert abs(ref - np.prod(f(xi, xj))) <= 1e-12


def test_single_qubit_closed_form(oracle):
    rng = np.random.default_rng(5)
    for reps in (1, 2, 3):
        for _ in range(5):
            a, b = rng.random(2) * PI
            ref = abs(np.vdot(_single_qubit_state(b, reps), _single_qubit_state(a, reps))) ** 2
            k_sv, _ = oracle.sv_kernel_pair(np.array([a]), np.array([b]), reps)
            K_mps, _ = oracle.mps_cross(np.array([[a]]), np.array([[b]]), reps)
            assert abs(k_sv - ref) <= 1e-13 and abs(K_mps[0, 0] - ref) <= 1e-13


# ---- structural facts: diagonal, symmetry, range, PSD ---------------------
@pytest.mark.parametrize("n,reps", [(6, 1), (6, 2), (6, 3), (40, 2), (120, 3)])
def test_gram_structure(oracle, n, reps):
    rng = np.random.default_rng(n + reps)
    X = _rand(rng, n, 24)
    K, LK = oracle.mps_gram(X, reps)
    Kc, _ = oracle.mps_cross(X, X, reps)  # both orders contracted separately
    assert np.all(np.abs(np.diag(Kc) - 1.0) <= 1e-12)
    assert np.max(np.abs(Kc - Kc.T)) <= 1e-12
    assert np.all(Kc >= 0.0) and np.all(Kc <= 1.0 + 1e-12)
    assert np.array_equal(K, K.T)
    assert np.min(np.linalg.eigvalsh(K)) >= -1e-12
    nz = K > 1e-300
    assert np.max(np.abs(np.log(K[nz]) - LK[nz])) <= 1e-9


def test_statevector_gram_psd(oracle):
    rng = np.random.default_rng(3)
    X = _rand(rng, 8, 32)
    K = oracle.sv_gram(X, 2)
    assert np.min(np.linalg.eigvalsh((K + K.T) / 2)) >= -1e-12
    assert np.all(np.abs(np.diag(K) - 1) <= 1e-12)


# ---- convention independence: RZ(2x) vs P(2x) differ by global phases ----
def test_phase_gate_invariance(oracle):
    rng = np.random.default_rng(9)
    for reps in (1, 2, 3):
        xi, xj = _rand(rng, 6, 2)
        k_rz, a_rz = oracle.sv_kernel_pair(xi, xj, reps)
        k_p, a_p = oracle.sv_kernel_pair(xi, xj, reps, oracle.PHASE_GATE)
        assert abs(k_rz - k_p) <= 1e-12


# ---- bond dimension: Schmidt ranks of exact states are <= 2^reps ----------
@pytest.mark.parametrize("reps", [1, 2, 3])
def test_schmidt_rank_bound(oracle, reps):
    n = 8
    x = np.random.default_rng(reps).random(n) * PI
    psi = oracle.sv_state(x, reps)
    ranks = []
    for cut in range(1, n):
        # qubit q is bit q: reshape as (high qubits, low qubits) at the cut
        M = psi.reshape(2 ** (n - cut), 2 ** cut)
        sv = np.linalg.svd(M, compute_uv=False)
        ranks.append(int((sv > 1e-10 * sv[0]).sum()))
    bound = [min(2 ** reps, 2 ** c, 2 ** (n - c)) for c in range(1, n)]
    assert all(r <= b for r, b in zip(ranks, bound)), (ranks, bound)
    assert max(ranks) == min(2 ** reps, 2 ** (n // 2))


def test_mps_reconstructs_state(oracle):
    # the closed-form MPS, multiplied out, equals the gate-by-gate state vector
    for reps in (1, 2, 3):
        n = 6
        x = np.random.default_rng(40 + reps).random(n) * PI
        A = oracle.mps_closed_form(x, reps)
        psi = oracle.sv_state(x, reps)
        for s in range(2 ** n):
            v = np.zeros(A.shape[2], complex)
            v[0] = 1.0
            for k in range(n):
                v = v @ A[k, (s >> k) & 1]
            assert abs(v[0] - psi[s]) <= 1e-12


# ---- large n: concentration and log-K consistency --------------------------
def test_large_n_concentration(oracle):
    rng = np.random.default_rng(11)
    X = np.where(rng.random((4, 784)) < 0.8, 0.0, (1 - rng.random((4, 784))) * PI)
    K, LK = oracle.mps_gram(X, 2)
    assert np.all(np.abs(np.diag(K) - 1) <= 1e-12)
    off = LK[~np.eye(4, dtype=bool)]
    assert np.all(off < np.log(1e-20))  # exponential concentration of off-diagonals (Sec. 4.2)


# ---- planted mistakes: each must break at least one pin -------------------
@pytest.mark.parametrize("mut", ["MUT_ZZ_SIGN", "MUT_DROP_SIGN", "MUT_NO_CONJ", "MUT_SHIFT_COUPLING"])
def test_planted_mistakes_are_caught(oracle, mut):
    flag = getattr(oracle, mut)
    rng = np.random.default_rng(123)
    n = 5
    xi, xj = _rand(rng, n, 2)
    caught = []
    # pin 1: O1 vs O2
    for reps in (1, 2):
        k_sv, _ = oracle.sv_kernel_pair(xi, xj, reps, flag)
        k_mps = oracle.mps_overlap(oracle.mps_closed_form(xi, reps, flag), oracle.mps_closed_form(xj, reps, flag),
                                   reps, flag)[0]
        caught.append(abs(k_sv - k_mps) > 1e-9)
    # pin 2: brute-force Ising sum at reps = 1
    S = ((np.arange(2 ** n)[:, None] >> np.arange(n)[None, :]) & 1).astype(float)
    amp = np.exp(-1j * (_ising_energy(xi, S) - _ising_energy(xj, S))).sum() / 2 ** n
    k_sv, _ = oracle.sv_kernel_pair(xi, xj, 1, flag)
    caught.append(abs(k_sv - abs(amp) ** 2) > 1e-9)
    # pin 2b: brute-force path sum at reps = 2 (both oracles)
    k_ref = abs(np.vdot(_reps2_state(xj), _reps2_state(xi))) ** 2
    k_sv, _ = oracle.sv_kernel_pair(xi, xj, 2, flag)
    K_mps, _ = oracle.mps_cross(xi[None], xj[None], 2, flag)
    caught.append(abs(k_sv - k_ref) > 1e-9 or abs(K_mps[0, 0] - k_ref) > 1e-9)
    # pin 3: diagonal of the MPS oracle
    caught.append(abs(oracle.mps_overlap(oracle.mps_closed_form(xi, 2, flag), oracle.mps_closed_form(xi, 2, flag), 2,
                                         flag)[0] - 1) > 1e-9)
    assert any(caught), mut


# ---- frozen fixtures (written by tests/golden/make_golden.py from the oracle) --
def test_golden_fixtures(oracle):
    import json
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "oracle_fixtures.json")
    g = json.load(open(path))
    c0 = g["cfg0_n8_r2_N16"]
    X = np.array(c0["X"])
    K, _ = oracle.mps_gram(X, c0["reps"])
    assert np.max(np.abs(K - np.array(c0["K"]))) <= 1e-12
    for p in g["pairs_n10"]["pairs"]:
        K2, _ = oracle.mps_cross(np.array([p["xi"]]), np.array([p["xj"]]), p["reps"])
        assert abs(K2[0, 0] - p["K"]) <= 1e-12


def test_inputs_generators():
    from paper_2405_02630_gb300 import inputs
    X = inputs.mnist_like_features(2000, 784, 2)
    z = (X == 0).mean()
    assert 0.79 < z < 0.81 and X.max() <= np.pi and X[X > 0].min() > 0
    U = inputs.uniform_features(100, 8, 0)
    assert U.min() >= 0 and U.max() < np.pi
    assert np.array_equal(inputs.uniform_features(4, 3, 7), inputs.uniform_features(4, 3, 7))
    jobs = inputs.batch_jobs()
    assert len(jobs) == 32 and all(64 <= X.shape[0] <= 1024 for X, _ in jobs)
