"""CPU model of the split-FP32 arithmetic of the reps = 3 four-thread kernel (gauged
Kronecker stages), in its operation order, with the exactness checks of the reps = 2
model: every hi*hi product and hi sum the kernel takes as exact must be a float32 value.

Per site (E_c stored with the signs T S^c . S^c T, components below U/4, hi on U 2^-11):
    Z[p1 + 2 q2] = E[2 q2] + M[p1] E[1 + 2 q2]   (rows with q2 = 1 re-split onto U 2^-10)
    Y[p1 + 2 p2] = Z[p1] + M[p2] Z[p1 + 2]        (Y_1 re-split onto U 2^-10)
    X_s = Y_0 + rho_s Y_1                         (all of X re-split onto U 2^-9)
    W[pp1 + 2 r2] = X[2 r2] + conj(M_j[pp1]) X[1 + 2 r2]   (r2 = 1 re-split onto U 2^-9)
    E'[pp1 + 2 pp2] = W[pp1] + conj(M_j[pp2]) W[pp1 + 2]
then E' is renormalised below 1/4 and re-split onto 2^-11.
"""
import numpy as np
import pytest

from paper_2405_02630_gb300 import inputs

from test_split_arithmetic import _Model, _gauged, f32


def _smac(M, hh, ll, w, V, conj_v):
    wh, wl, wf = w
    vh, vl = (np.conj(V[0]), np.conj(V[1])) if conj_v else V
    hr = M.exact(M.exact(hh.real + wh.real * vh.real) - wh.imag * vh.imag)
    hi = M.exact(M.exact(hh.imag + wh.real * vh.imag) + wh.imag * vh.real)
    lr = M.fma(wf.imag, -vl.imag, M.fma(wf.real, vl.real, M.fma(wl.imag, -vh.imag, M.fma(wl.real, vh.real, ll.real))))
    li = M.fma(wf.imag, vl.real, M.fma(wf.real, vl.imag, M.fma(wl.imag, vh.real, M.fma(wl.real, vh.imag, ll.imag))))
    return hr + 1j * hi, lr + 1j * li


def _split(M, hh, ll, grid):
    v = f32(hh.real + ll.real) + 1j * f32(hh.imag + ll.imag)
    xh = M.rnd(v.real, grid) + 1j * M.rnd(v.imag, grid)
    xl = f32(M.exact(hh.real - xh.real) + ll.real) + 1j * f32(M.exact(hh.imag - xh.imag) + ll.imag)
    return xh, xl, v


def _full(h, l):
    return h, l, f32(h.real + l.real) + 1j * f32(h.imag + l.imag)


def _contract(Xa, Xb):
    M = _Model()
    (ai, bi), (aj, bj) = _gauged(Xa), _gauged(Xb)
    P, n1 = ai[0].shape
    t3 = lambda q: -1.0 if q == 3 else 1.0
    sS = lambda q: -1.0 if q >= 2 else 1.0
    Eh = np.zeros((2, 4, 4, P), complex)
    El = np.zeros((2, 4, 4, P), complex)
    Eh[0, 0, 0] = 1.0
    U = 8.0  # E = e_0 e_0^T: largest component 1 < U / 4
    L = np.full(P, 3.0)
    for k in range(n1):
        A = [(ai[0][:, k], ai[1][:, k]), (bi[0][:, k], bi[1][:, k])]
        B = [(aj[0][:, k], aj[1][:, k]), (bj[0][:, k], bj[1][:, k])]
        R = []
        for s in range(2):
            (uh, ul), (wh, wl) = A[s], B[s]
            hr = M.exact(uh.real * wh.real + uh.imag * wh.imag)
            hi = M.exact(uh.imag * wh.real - uh.real * wh.imag)
            fr, fi = f32(uh.real + ul.real), f32(uh.imag + ul.imag)
            lr = M.fma(ul.real, wh.real, M.fma(ul.imag, wh.imag, M.fma(fr, wl.real, f32(fi * wl.imag))))
            li = M.fma(ul.real, -wh.imag, M.fma(ul.imag, wh.real, M.fma(fr, -wl.imag, f32(fi * wl.real))))
            R.append(_split(M, hr + 1j * hi, lr + 1j * li, 2.0 ** -11)[:2])
        Y = {}
        for c in range(2):
            for r in range(4):
                Z = {}
                for q2 in range(2):
                    w = _full(Eh[c, 1 + 2 * q2, r], El[c, 1 + 2 * q2, r])
                    for p1 in range(2):
                        hh, ll = _smac(M, Eh[c, 2 * q2, r], El[c, 2 * q2, r], w, A[p1], False)
                        Z[p1 + 2 * q2] = _split(M, hh, ll, U * 2.0 ** -10) if q2 else (hh, ll)
                for p2 in range(2):
                    for p1 in range(2):
                        hh, ll = _smac(M, Z[p1][0], Z[p1][1], Z[p1 + 2], A[p2], False)
                        Y[c, p1 + 2 * p2, r] = _split(M, hh, ll, U * 2.0 ** -10) if c else (hh, ll)
        Nh = np.zeros((2, 4, 4, P), complex)
        Nl = np.zeros((2, 4, 4, P), complex)
        for s in range(2):
            Xs = {}
            for p in range(4):
                for r in range(4):
                    hh, ll = _smac(M, Y[0, p, r][0], Y[0, p, r][1], Y[1, p, r], R[s], False)
                    Xs[p, r] = _split(M, hh, ll, U * 2.0 ** -9)
            for p in range(4):
                W = {}
                for r2 in range(2):
                    w = _full(Xs[p, 1 + 2 * r2][0], Xs[p, 1 + 2 * r2][1])
                    for pp1 in range(2):
                        hh, ll = _smac(M, Xs[p, 2 * r2][0], Xs[p, 2 * r2][1], w, B[pp1], True)
                        W[pp1 + 2 * r2] = _split(M, hh, ll, U * 2.0 ** -9) if r2 else (hh, ll)
                for pp2 in range(2):
                    for pp1 in range(2):
                        Nh[s, p, pp1 + 2 * pp2], Nl[s, p, pp1 + 2 * pp2] = _smac(
                            M, W[pp1][0], W[pp1][1], W[pp1 + 2], B[pp2], True)
        V = f32(Nh.real + Nl.real) + 1j * f32(Nh.imag + Nl.imag)
        m = np.max(np.maximum(np.abs(V.real), np.abs(V.imag)).reshape(-1, P), axis=0)
        e = np.frexp(m)[1] + 2  # components below 1/4 after scaling by 2^-e
        sc = np.ldexp(1.0, -e)
        for s in range(2):
            for p in range(4):
                for pp in range(4):
                    sg = t3(p) * t3(pp) * ((sS(p) * sS(pp)) if s else 1.0)
                    f = f32(V[s, p, pp].real * sc * sg) + 1j * f32(V[s, p, pp].imag * sc * sg)
                    h = M.rnd(f.real, 2.0 ** -11) + 1j * M.rnd(f.imag, 2.0 ** -11)
                    lr = M.fma(Nl[s, p, pp].real, sc * sg, M.exact(Nh[s, p, pp].real * sc * sg - h.real))
                    li = M.fma(Nl[s, p, pp].imag, sc * sg, M.exact(Nh[s, p, pp].imag * sc * sg - h.imag))
                    Eh[s, p, pp], El[s, p, pp] = h, lr + 1j * li
        L = L + e - 3
        U = 1.0
    amp = Eh[0, 0, 0] + El[0, 0, 0]
    return np.abs(amp) ** 2 * 2.0 ** (2 * L), M.inexact


@pytest.fixture(scope="module")
def pairs3(oracle):
    base = inputs.mnist_like_features(12, 784, 31)
    pert = inputs.near_duplicates(base, 32)
    ra, rb = inputs.mnist_like_features(12, 784, 35), inputs.mnist_like_features(12, 784, 36)
    idx = np.arange(12)
    K1, _ = oracle.mps_pairs(base, pert, idx, idx, 3)
    K2, _ = oracle.mps_pairs(ra, rb, idx, idx, 3)
    return (base, pert, K1), (ra, rb, K2)


def test_reps3_split_arithmetic_is_exact_and_accurate(pairs3):
    (base, pert, K1), (ra, rb, K2) = pairs3
    k1, bad1 = _contract(base, pert)
    k2, bad2 = _contract(ra, rb)
    assert bad1 == 0 and bad2 == 0, f"inexact hi operations: {bad1}, {bad2}"
    assert np.max(np.abs(k1 - K1)) <= 5e-8
    assert K2.max() < 1e-150 and np.max(np.abs(np.log(k2 / K2))) <= 1e-5
