"""CPU checks of the site-tensor structure the CUDA contraction relies on, on the
oracle's dense closed-form tensors (oracle.mps_closed_form: A[k, sigma, t, u], layer
m of a bond index in bit m-1, so the last layer is the HIGH bit there).

1. The last layer is diagonal: A^sigma[t][u] = 0 unless the last-layer bit of u is sigma.
2. The left neighbour's last-layer spin c enters only through the last ZZ phase:
   rows with c = 1 equal the rows with c = 0 times exp(2 i theta z(sigma)).
3. At reps = 2 every entry is +-1/2 times 1, T^2, P^2 or P^2 T^2 or a conjugate
   (P = exp(-i x_k), T = exp(-i theta_{k-1})), in the pattern the phase-form records
   encode, and contracting with that pattern reproduces the state-vector kernel; at
   reps = 3 every entry is +-2^{-3/2} P^A T^B or a conjugate, in the pattern of the
   split-FP32 records at reps = 3.
4. The gauged form of the split-FP32 records at reps = 2: after the diagonal change of
   bond basis that makes row t = 0 of every site tensor one, both blocks of site k are
   [[1, 1], [alpha_k, beta_k]] and the c = 1 rows are r'_s diag(1, -1) times the c = 0
   rows with r'_0 = alpha_k, r'_1 = beta_k; contracting with those tensors plus one
   virtual site reproduces the state-vector kernel, also where K is tiny.
5. The same change of basis at reps = 3 gives the same two phases per site: both
   blocks equal (-1)^{q1 q2} M[q1][p1] M[q2][p2] with M = [[1, 1], [alpha_k, beta_k]]
   (a signed Kronecker square of the reps = 2 block) and the c = 1 rows are r'_s
   diag(1, 1, -1, -1) times the c = 0 rows, r'_0 = alpha_k, r'_1 = beta_k.
"""
import numpy as np
import pytest

from paper_2405_02630_gb300 import inputs


def _theta(x):
    th = np.zeros_like(x)
    th[1:] = (np.pi - x[:-1]) * (np.pi - x[1:])
    return th


@pytest.mark.parametrize("reps", [1, 2, 3])
def test_last_layer_diagonal_and_row_factorisation(oracle, reps):
    n = 7
    x = inputs.uniform_features(1, n, 300 + reps)[0]
    A = oracle.mps_closed_form(x, reps)
    chi, H = 2 ** reps, 2 ** (reps - 1)
    th = _theta(x)
    for k in range(n):
        for sigma in range(2):
            for u in range(chi):
                if (u >> (reps - 1)) != sigma and k < n - 1:
                    assert np.all(A[k, sigma, :, u] == 0)
            if k == 0:
                continue
            r = np.exp(2j * th[k] * (1 - 2 * sigma))
            rows0, rows1 = A[k, sigma, :H, :], A[k, sigma, H:, :]  # last-layer bit c = 0 / 1
            assert np.max(np.abs(rows1 - r * rows0)) <= 1e-14


def test_reps2_phase_form(oracle):
    n = 9
    x = inputs.mnist_like_features(1, n, 310)[0]
    A = oracle.mps_closed_form(x, 2)
    th = _theta(x)
    for k in range(n - 1):  # the oracle sums the last site's right bond
        P2, T2 = np.exp(-2j * x[k]), np.exp(-2j * th[k])
        V0, V1, V2 = T2, P2, P2 * T2
        # blocks a_0s[q][p] = A[s][t = (q, c = 0)][u = (p, s)]; in the oracle's bit order
        # layer 1 is bit 0 and layer 2 (the last) bit 1, so t = q + 2c and u = p + 2s.
        # Site 0 has only t = 0 (its other rows meet a zero environment in the contraction).
        rows = 1 if k == 0 else 2
        for s, want in ((0, [[V2, 1], [V1, V0]]), (1, [[1, -np.conj(V2)], [np.conj(V0), -np.conj(V1)]])):
            blk = np.array([[A[k, s, q, p + 2 * s] for p in range(2)] for q in range(rows)])
            assert np.max(np.abs(blk - 0.5 * np.array(want)[:rows])) <= 1e-14, (k, s)


def test_reps2_phase_form_contraction(oracle):
    """Contract two points with the phase-form update (open last bond, amplitude = sum of
    all entries) and compare with the state-vector kernel."""
    n = 8
    X = inputs.uniform_features(2, n, 320)
    def ph(x):
        th = _theta(x)
        return np.exp(-2j * th), np.exp(-2j * x), np.exp(-2j * (x + th))
    (V0, V1, V2), (W0, W1, W2) = ph(X[0]), ph(X[1])
    E = [np.zeros((2, 2), complex), np.zeros((2, 2), complex)]
    E[0][0, 0] = 1.0
    for k in range(n):
        a = [0.5 * np.array([[V2[k], 1], [V1[k], V0[k]]]),
             0.5 * np.array([[1, -np.conj(V2[k])], [np.conj(V0[k]), -np.conj(V1[k])]])]
        b = [0.5 * np.array([[W2[k], 1], [W1[k], W0[k]]]),
             0.5 * np.array([[1, -np.conj(W2[k])], [np.conj(W0[k]), -np.conj(W1[k])]])]
        rho0 = np.conj(V0[k]) * W0[k]
        rho = [rho0, np.conj(rho0)]
        E = [a[s].T @ (E[0] + rho[s] * E[1]) @ np.conj(b[s]) for s in range(2)]
    K = abs(E[0].sum() + E[1].sum()) ** 2
    Ko, _ = oracle.sv_kernel_pair(X[0], X[1], 2)
    assert abs(K - Ko) <= 1e-13


def test_reps3_phase_form(oracle):
    """At reps = 3 every entry is +-2^{-3/2} P^A T^B (A, B in {3, 1, -1}) or a conjugate:
    with q = 2 q1 + q2, p = 2 p1 + p2 (layer 1 the high bit) and W[ia][ib] =
    2^{-3/2} P^{3 - 2 ia} T^{3 - 2 ib}, a_00[q][p] = (-1)^{p1 p2} W[p1 + p2][(q1^p1) + (q2^p2)]
    and a_01[q][p] = (-1)^{p1 p2 + p2} conj(W[2 - ia][2 - ib])."""
    n = 7
    x = inputs.uniform_features(1, n, 333)[0]
    A = oracle.mps_closed_form(x, 3)  # oracle bit order: layer m in bit m - 1
    th = _theta(x)
    for k in range(1, n - 1):
        P, T = np.exp(-1j * x[k]), np.exp(-1j * th[k])
        W = np.array([[2 ** -1.5 * P ** a * T ** b for b in (3, 1, -1)] for a in (3, 1, -1)])
        for s in range(2):
            for q in range(4):
                for p in range(4):
                    q1, q2, p1, p2 = q >> 1, q & 1, p >> 1, p & 1
                    val = A[k, s, q1 + 2 * q2, p1 + 2 * p2 + 4 * s]
                    ia, ib = p1 + p2, (q1 ^ p1) + (q2 ^ p2)
                    pred = ((-1) ** (p1 * p2) * W[ia, ib] if s == 0
                            else (-1) ** (p1 * p2 + p2) * np.conj(W[2 - ia, 2 - ib]))
                    assert abs(val - pred) <= 1e-14, (k, s, q, p)


def _gauged_alpha_beta(x):
    """alpha_k = conj(V2^{k-1} V0^k), beta_k = conj(V2^{k-1}) V0^k for sites 0..n (site n
    virtual, with V0^n = 1); V0 = T^2 and V2 = P^2 T^2 of the phase form, V2^{-1} = 1."""
    n = len(x)
    th = np.concatenate([_theta(x), [0.0]])
    V0 = np.exp(-2j * th)
    V2p = np.concatenate([[1.0], np.exp(-2j * (x + th[:n]))])
    return np.conj(V2p) * np.conj(V0), np.conj(V2p) * V0


def test_reps2_gauged_form(oracle):
    """Gauge the oracle's tensors site by site: column u of site k is divided by its row-0
    entry and row t multiplied by l_t = A_{k-1}[0][u = t] / A_{k-1}[0][u = 0] (the basis
    change the previous site left on the bond), then compare with the gauged pattern."""
    n = 9
    x = inputs.mnist_like_features(1, n, 340)[0]
    x[3] = 0.7  # a nonzero feature next to zeros, whatever the seed gives
    A = oracle.mps_closed_form(x, 2)  # bit order: t = q + 2c, u = p + 2s
    alpha, beta = _gauged_alpha_beta(x)
    S = np.diag([1.0, -1.0])
    row0 = lambda k, u: A[k, u >> 1, 0, u]  # row t = 0, column u (sigma = last-layer bit s of u)
    for k in range(1, n - 1):
        ell = np.array([row0(k - 1, t) / row0(k - 1, 0) for t in range(4)])
        for s in range(2):
            blk = {c: np.array([[ell[q + 2 * c] * A[k, s, q + 2 * c, p + 2 * s] / row0(k, p + 2 * s)
                                 for p in range(2)] for q in range(2)]) for c in range(2)}
            a0 = np.array([[1, 1], [alpha[k], beta[k]]])
            assert np.max(np.abs(blk[0] - a0)) <= 1e-13, (k, s)
            r = alpha[k] if s == 0 else beta[k]
            assert np.max(np.abs(blk[1] - r * S @ a0)) <= 1e-13, (k, s)


@pytest.mark.parametrize("n,seed", [(2, 341), (7, 342), (12, 343)])
def test_reps2_gauged_contraction(oracle, n, seed):
    """E_{k+1} blocks: G_s = E_0 + rho_s E_1 (rho_0 = alpha_i conj(alpha_j), rho_1 = beta_i
    conj(beta_j)), E'_s = a^T G_s conj(b) with E_1 kept as S E_1 S; after the virtual site
    n the amplitude is E_0[0][0] up to a phase, times 2^-2 per real site."""
    X = np.concatenate([inputs.uniform_features(3, n, seed), inputs.mnist_like_features(1, n, seed)])
    S = np.diag([1.0, -1.0])
    for i, j in ((0, 1), (1, 2), (3, 0), (2, 2)):
        (ai, bi), (aj, bj) = _gauged_alpha_beta(X[i]), _gauged_alpha_beta(X[j])
        E = [np.zeros((2, 2), complex), np.zeros((2, 2), complex)]
        E[0][0, 0] = 1.0
        for k in range(n + 1):
            a = np.array([[1, 1], [ai[k], bi[k]]])
            b = np.array([[1, 1], [aj[k], bj[k]]])
            rho = [ai[k] * np.conj(aj[k]), bi[k] * np.conj(bj[k])]
            E = [a.T @ (E[0] + rho[s] * E[1]) @ np.conj(b) for s in range(2)]
            E[1] = S @ E[1] @ S
        K = abs(E[0][0, 0]) ** 2 * 2.0 ** (-4 * n)
        Ko, _ = oracle.sv_kernel_pair(X[i], X[j], 2)
        assert abs(K - Ko) <= 1e-13 and abs(K / Ko - 1) <= 1e-11, (n, i, j, K, Ko)


def test_reps3_gauged_form_is_a_kronecker_square(oracle):
    """Row-0 gauge of the oracle's reps = 3 tensors (oracle bit order: q = q1 + 2 q2 with
    q1 layer 1, the last layer in bit 2 of t and u): both blocks of site k are the signed
    Kronecker square of the reps = 2 block [[1, 1], [alpha_k, beta_k]] with the same
    alpha_k, beta_k, and the c = 1 rows carry r'_s diag(1, 1, -1, -1)."""
    n = 9
    x = inputs.uniform_features(1, n, 350)[0]
    x[4] = 0.0  # a blank feature, as in MNIST-like data
    A = oracle.mps_closed_form(x, 3)
    alpha, beta = _gauged_alpha_beta(x)
    row0 = lambda k, u: A[k, u >> 2, 0, u]
    S = np.diag([1.0, 1.0, -1.0, -1.0])
    for k in range(1, n - 1):
        ell = np.array([row0(k - 1, t) / row0(k - 1, 0) for t in range(8)])
        M = np.array([[1, 1], [alpha[k], beta[k]]])
        kron = np.array([[(-1) ** ((q & 1) * (q >> 1)) * M[q & 1, p & 1] * M[q >> 1, p >> 1] for p in range(4)]
                         for q in range(4)])
        for s in range(2):
            blk = {c: np.array([[ell[q + 4 * c] * A[k, s, q + 4 * c, p + 4 * s] / row0(k, p + 4 * s)
                                 for p in range(4)] for q in range(4)]) for c in range(2)}
            assert np.max(np.abs(blk[0] - kron)) <= 1e-13, (k, s)
            r = alpha[k] if s == 0 else beta[k]
            assert np.max(np.abs(blk[1] - r * S @ kron)) <= 1e-13, (k, s)


@pytest.mark.parametrize("n,seed", [(2, 361), (6, 362), (9, 363)])
def test_reps3_gauged_contraction(oracle, n, seed):
    """The reps = 3 update of the four-thread engine: with the row signs T = diag(1, 1, 1, -1)
    and S = diag(1, 1, -1, -1) folded into the stored environment Ev_c = T S^c E_c S^c T,
    Y_c = (M_i x M_i)^T Ev_c in two 2 x 2 stages, X_s = Y_0 + rho_s Y_1, E'_s = X_s
    conj(M_j x M_j) in two stages; after the virtual site K = |E_0[0][0]|^2 2^(-6n)."""
    X = np.concatenate([inputs.uniform_features(3, n, seed), inputs.mnist_like_features(1, n, seed)])
    T = np.array([1.0, 1.0, 1.0, -1.0])
    Sg = np.array([1.0, 1.0, -1.0, -1.0])

    def rows(Mv, E):  # (M x M)^T applied to the row index q = q1 + 2 q2 of E, as two stages
        a, b = Mv
        Z = np.stack([E[0] + a * E[1], E[0] + b * E[1], E[2] + a * E[3], E[2] + b * E[3]])
        return np.stack([Z[0] + a * Z[2], Z[1] + a * Z[3], Z[0] + b * Z[2], Z[1] + b * Z[3]])

    for i, j in ((0, 1), (2, 3), (1, 1)):
        (ai, bi), (aj, bj) = _gauged_alpha_beta(X[i]), _gauged_alpha_beta(X[j])
        Ev = [np.zeros((4, 4), complex), np.zeros((4, 4), complex)]
        Ev[0][0, 0] = 1.0
        for k in range(n + 1):
            Y = [rows((ai[k], bi[k]), Ev[c]) for c in range(2)]
            rho = [ai[k] * np.conj(aj[k]), bi[k] * np.conj(bj[k])]
            new = []
            for s in range(2):
                Xs = Y[0] + rho[s] * Y[1]
                Ep = rows((np.conj(aj[k]), np.conj(bj[k])), Xs.T).T  # columns, conjugated M_j
                sg = np.outer(T, T) * (np.outer(Sg, Sg) if s else 1.0)
                new.append(sg * Ep)
            Ev = new
        K = abs(Ev[0][0, 0]) ** 2 * 2.0 ** (-6 * n)
        Ko, _ = oracle.sv_kernel_pair(X[i], X[j], 3)
        assert abs(K - Ko) <= 1e-13 and abs(K / Ko - 1) <= 1e-11, (n, i, j, K, Ko)
