"""Python front end of the plain FP64 CPU oracle (``qsvm_oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py`` (its CPU-baseline and reference legs).  The product package never
imports this module, and this module never imports the product package.

It computes the quantum kernel of arXiv 2405.02630, Sec. 2 Eq. 3-4,
K(x_i, x_j) = |<psi(x_j)|psi(x_i)>|^2, for the linear-chain feature map of
Sec. 3.2, in two independent ways:

* ``sv_*``  -- O1, a gate-by-gate state vector (Algorithm 1's recipe), n <= 20;
* ``mps_*`` -- O2, the closed-form path-sum MPS contracted site by site
  (the tensor-network route of Algorithms 2-3), any n.

The numerical work is plain C (``qsvm_oracle.c``) compiled with gcc; this file
only marshals numpy arrays.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qsvm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

NO_ENTANGLER = 1
PHASE_GATE = 2
MUT_ZZ_SIGN = 4
MUT_DROP_SIGN = 8
MUT_NO_CONJ = 16
MUT_SHIFT_COUPLING = 32

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` next to its source (gcc, OpenMP)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB)
            dp = ctypes.POINTER(ctypes.c_double)
            i64p = ctypes.POINTER(ctypes.c_int64)
            c_int, i64 = ctypes.c_int, ctypes.c_int64
            L.qo_sv_state.argtypes = [dp, c_int, c_int, c_int, dp]
            L.qo_sv_state.restype = c_int
            L.qo_sv_kernel_pair.argtypes = [dp, dp, c_int, c_int, c_int, dp]
            L.qo_sv_kernel_pair.restype = ctypes.c_double
            L.qo_sv_cross.argtypes = [dp, i64, dp, i64, c_int, c_int, c_int, dp, c_int]
            L.qo_sv_cross.restype = c_int
            L.qo_mps_closed_form.argtypes = [dp, c_int, c_int, c_int, dp]
            L.qo_mps_closed_form.restype = c_int
            L.qo_mps_overlap.argtypes = [dp, dp, c_int, c_int, c_int, dp, dp, dp]
            L.qo_mps_overlap.restype = ctypes.c_double
            L.qo_mps_cross.argtypes = [dp, i64, dp, i64, c_int, c_int, c_int, c_int, dp, i64, dp, i64, c_int]
            L.qo_mps_cross.restype = c_int
            L.qo_mps_pairs.argtypes = [dp, dp, i64p, i64p, i64, c_int, c_int, c_int, dp, dp, c_int]
            L.qo_mps_pairs.restype = c_int
            i8p = ctypes.POINTER(ctypes.c_byte)
            L.qo_svc_fit.argtypes = [dp, ctypes.c_longlong, i64p, i8p, ctypes.c_longlong, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_longlong, dp, dp]
            L.qo_svc_fit.restype = ctypes.c_longlong
            L.qo_svc_decision.argtypes = [dp, ctypes.c_longlong, i64p, ctypes.c_longlong, dp, i8p, ctypes.c_double,
                                          ctypes.c_longlong, dp]
            L.qo_svc_decision.restype = None
            L.qo_max_threads.argtypes = []
            L.qo_max_threads.restype = c_int
            _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def max_threads() -> int:
    return int(lib().qo_max_threads())


# ------------------------------------------------------------------ O1 ---
def sv_state(x, reps: int, flags: int = 0) -> np.ndarray:
    """U(x)|0^n> as a complex128 vector of length 2^n (qubit q is bit q)."""
    x = _f64(x)
    n = x.shape[0]
    out = np.zeros(2 ** n, dtype=np.complex128)
    rc = lib().qo_sv_state(_dp(x), n, reps, flags, _dp(out.view(np.float64)))
    if rc != 0:
        raise ValueError(f"qo_sv_state failed ({rc})")
    return out


def sv_kernel_pair(xi, xj, reps: int, flags: int = 0):
    """Algorithm 1 recipe for one pair: returns (K, amp) with amp = <0|U^dag(x_j) U(x_i)|0>."""
    xi, xj = _f64(xi), _f64(xj)
    amp = np.zeros(2)
    k = lib().qo_sv_kernel_pair(_dp(xi), _dp(xj), xi.shape[0], reps, flags, _dp(amp))
    if k < 0:
        raise ValueError("qo_sv_kernel_pair failed")
    return float(k), complex(amp[0], amp[1])


def sv_cross(Xa, Xb, reps: int, flags: int = 0, threads: int = 0) -> np.ndarray:
    Xa, Xb = _f64(Xa), _f64(Xb)
    na, n = Xa.shape
    nb = Xb.shape[0]
    K = np.zeros((na, nb))
    rc = lib().qo_sv_cross(_dp(Xa), na, _dp(Xb), nb, n, reps, flags, _dp(K), threads)
    if rc != 0:
        raise ValueError(f"qo_sv_cross failed ({rc})")
    return K


def sv_gram(X, reps: int, flags: int = 0, threads: int = 0) -> np.ndarray:
    return sv_cross(X, X, reps, flags, threads)


# ------------------------------------------------------------------ O2 ---
def mps_closed_form(x, reps: int, flags: int = 0) -> np.ndarray:
    """Dense closed-form site tensors A[k, sigma, t, u] (complex128, chi = 2^reps)."""
    x = _f64(x)
    n = x.shape[0]
    chi = 2 ** reps
    A = np.zeros((n, 2, chi, chi), dtype=np.complex128)
    rc = lib().qo_mps_closed_form(_dp(x), n, reps, flags, _dp(A.view(np.float64)))
    if rc != 0:
        raise ValueError(f"qo_mps_closed_form failed ({rc})")
    return A


def mps_overlap(A, B, reps: int, flags: int = 0):
    """K = |<B|A>|^2 of two dense MPS; returns (K, lnK, amp_scaled, ln_scale)."""
    A = np.ascontiguousarray(A, dtype=np.complex128)
    B = np.ascontiguousarray(B, dtype=np.complex128)
    n = A.shape[0]
    lk = np.zeros(1)
    amp = np.zeros(2)
    ls = np.zeros(1)
    k = lib().qo_mps_overlap(_dp(A.view(np.float64)), _dp(B.view(np.float64)), n, reps, flags, _dp(lk), _dp(amp),
                             _dp(ls))
    return float(k), float(lk[0]), complex(amp[0], amp[1]), float(ls[0])


def mps_cross(Xa, Xb, reps: int, flags: int = 0, threads: int = 0):
    """Cross kernel K[a, b] = |<psi(Xb[b])|psi(Xa[a])>|^2 and ln K."""
    Xa, Xb = _f64(Xa), _f64(Xb)
    na, n = Xa.shape
    nb = Xb.shape[0]
    K = np.zeros((na, nb))
    LK = np.zeros((na, nb))
    rc = lib().qo_mps_cross(_dp(Xa), na, _dp(Xb), nb, n, reps, flags, 0, _dp(K), nb, _dp(LK), nb, threads)
    if rc != 0:
        raise ValueError(f"qo_mps_cross failed ({rc})")
    return K, LK


def mps_gram(X, reps: int, flags: int = 0, threads: int = 0):
    """Symmetric Gram: contracts a <= b (diagonal included) and mirrors."""
    X = _f64(X)
    N, n = X.shape
    K = np.zeros((N, N))
    LK = np.zeros((N, N))
    rc = lib().qo_mps_cross(_dp(X), N, _dp(X), N, n, reps, flags, 1, _dp(K), N, _dp(LK), N, threads)
    if rc != 0:
        raise ValueError(f"qo_mps_cross failed ({rc})")
    return K, LK


def mps_pairs(Xa, Xb, ia, ib, reps: int, flags: int = 0, threads: int = 0):
    """K and ln K for explicit pairs (Xa[ia[p]], Xb[ib[p]])."""
    Xa, Xb = _f64(Xa), _f64(Xb)
    ia = np.ascontiguousarray(ia, dtype=np.int64)
    ib = np.ascontiguousarray(ib, dtype=np.int64)
    n = Xa.shape[1]
    K = np.zeros(ia.shape[0])
    LK = np.zeros(ia.shape[0])
    i64p = ctypes.POINTER(ctypes.c_int64)
    rc = lib().qo_mps_pairs(_dp(Xa), _dp(Xb), ia.ctypes.data_as(i64p), ib.ctypes.data_as(i64p), ia.shape[0], n, reps,
                            flags, _dp(K), _dp(LK), threads)
    if rc != 0:
        raise ValueError(f"qo_mps_pairs failed ({rc})")
    return K, LK


# ----------------------------------------------------------------- SVC ---
def svc_fit(K, y, C: float = 1.0, tol: float = 1e-8, max_iter: int = 1_000_000, idx=None):
    """Binary C-SVC dual on a precomputed kernel by SMO (maximal violating pair).
    Returns (alpha, b, iterations)."""
    K = np.ascontiguousarray(K, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.int8)
    n = y.shape[0] if idx is None else len(idx)
    ip = None
    if idx is not None:
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        ip = idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    alpha = np.zeros(n)
    b = np.zeros(1)
    it = lib().qo_svc_fit(_dp(K), K.shape[1], ip, y.ctypes.data_as(ctypes.POINTER(ctypes.c_byte)), n, C, tol,
                          max_iter, _dp(alpha), _dp(b))
    if it < 0:
        raise ValueError("qo_svc_fit failed")
    return alpha, float(b[0]), int(it)


def svc_decision(Kx, alpha, y, b: float, idx=None):
    Kx = np.ascontiguousarray(Kx, dtype=np.float64)
    y = np.ascontiguousarray(y, dtype=np.int8)
    alpha = np.ascontiguousarray(alpha, dtype=np.float64)
    ip = None
    if idx is not None:
        idx = np.ascontiguousarray(idx, dtype=np.int64)
        ip = idx.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    f = np.zeros(Kx.shape[0])
    lib().qo_svc_decision(_dp(Kx), Kx.shape[1], ip, Kx.shape[0], _dp(alpha),
                          y.ctypes.data_as(ctypes.POINTER(ctypes.c_byte)), b, alpha.shape[0], _dp(f))
    return f
