"""Thin ctypes binding of libqsvm (include/qsvm.h), same entry-point names.

Argument marshalling only: every step of the computation runs in the library's
CUDA kernels.  PyTorch supplies device memory and streams.  There is no CPU
fallback: if libqsvm.so is missing or cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libqsvm.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "qsvm.h")

QSVM_OK = 0
QSVM_ERR_ARG = -1
QSVM_ERR_CHI = -2
QSVM_ERR_CUDA = -3
QSVM_ERR_TIMEOUT = -4
QSVM_ERR_UNIMPLEMENTED = -5
QSVM_ERR_WORKSPACE = -6

QSVM_FP64 = 0
QSVM_FP32 = 1
QSVM_FP32_SPLIT = 2
PRECISIONS = {"fp64": QSVM_FP64, "fp32": QSVM_FP32, "fp32_split": QSVM_FP32_SPLIT}


class QsvmError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"qsvm error {code}: {msg}")
        self.code = code


_lock = threading.Lock()
_lib = None

_i32, _i64, _sz, _vp, _dp = ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p


class QsvmJob(ctypes.Structure):
    """Mirror of struct qsvm_job (include/qsvm.h)."""
    _fields_ = [("mps", ctypes.c_void_p), ("n_points", ctypes.c_int64), ("n_qubits", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("K", ctypes.c_void_p), ("ldk", ctypes.c_int64),
                ("logK", ctypes.c_void_p), ("ldl", ctypes.c_int64)]


class QsvmSvcProblem(ctypes.Structure):
    """Mirror of struct qsvm_svc_problem (include/qsvm.h)."""
    _fields_ = [("idx", ctypes.c_void_p), ("y", ctypes.c_void_p), ("n", ctypes.c_int64), ("alpha", ctypes.c_void_p)]


_SIGS = {
    "qsvm_mps_record_bytes": (_sz, [_i32, _i32]),
    "qsvm_mps_point_bytes": (_sz, [_i32, _i32, _i32]),
    "qsvm_mps_bytes": (_sz, [_i32, _i32, _i64, _i32]),
    "qsvm_build_mps": (_i32, [_dp, _i64, _i32, _i32, _i32, _vp, _sz, _vp]),
    "qsvm_kernel_gram": (_i32, [_vp, _i64, _i32, _i32, _i32, _dp, _i64, _dp, _i64, _vp]),
    "qsvm_kernel_cross": (_i32, [_vp, _i64, _vp, _i64, _i32, _i32, _i32, _dp, _i64, _dp, _i64, _vp]),
    "qsvm_gram_host_workspace_bytes": (_sz, [_i64, _i32, _i32, _i32, _i32]),
    "qsvm_gram_host": (_i32, [_dp, _i64, _i32, _i32, _i32, _dp, _i64, _dp, _i64, _vp, _sz, _vp]),
    "qsvm_cross_host_workspace_bytes": (_sz, [_i64, _i64, _i32, _i32, _i32, _i32]),
    "qsvm_cross_host": (_i32, [_dp, _i64, _dp, _i64, _i32, _i32, _i32, _dp, _i64, _dp, _i64, _vp, _sz, _vp]),
    "qsvm_gram_tile_dim": (_i32, [_i32, _i32]),
    "qsvm_gram_num_tiles": (_i64, [_i64, _i32, _i32]),
    "qsvm_gram_partition": (_i32, [_i64, _i32, _i32, _i32, _i32, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
    "qsvm_gram_tile_coords": (_i32, [_i64, _i32, _i32, _i64, ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
    "qsvm_gram_tile_list": (_i32, [_i64, _i32, _i32, _i64, _i64, _vp, _vp]),
    "qsvm_kernel_gram_tiles": (_i32, [_vp, _i64, _i32, _i32, _i32, _i64, _i64, _dp, _i64, _dp, _i64, _vp]),
    "qsvm_batch_workspace_bytes": (_sz, [_i32]),
    "qsvm_kernel_batch": (_i32, [ctypes.POINTER(QsvmJob), _i32, _i32, _i32, _vp, _sz, _vp]),
    "qsvm_kernel_batch_noalloc": (_i32, [ctypes.POINTER(QsvmJob), _i32, _i32, _i32, _vp]),
    "qsvm_batch_plan_create": (_i32, [ctypes.POINTER(QsvmJob), _i32, _i32, _i32, _vp, _sz,
                                      ctypes.POINTER(ctypes.c_void_p)]),
    "qsvm_batch_plan_launch": (_i32, [_vp, _vp]),
    "qsvm_batch_plan_destroy": (_i32, [_vp]),
    "qsvm_num_configs": (_i32, []),
    "qsvm_config_info": (_i32, [_i32, _i32, _i32, ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
    "qsvm_config_tile": (_i32, [_i32, _i32, _i32, ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
    "qsvm_set_config": (_i32, [_i32, _i32, _i32]),
    "qsvm_get_config": (_i32, [_i32, _i32]),
    "qsvm_autotune": (_i32, [_vp, _i64, _i32, _i32, _i32, _dp, _i64, _vp, ctypes.POINTER(_i32),
                             ctypes.POINTER(ctypes.c_float)]),
    "qsvm_device_status": (_i32, [_vp, _i32, ctypes.POINTER(_i32)]),
    "qsvm_selftest_wait_timeout": (_i32, [_i64, _vp]),
    "qsvm_sv_workspace_bytes": (_sz, [_i64, _i32]),
    "qsvm_svc_workspace_bytes": (_sz, [ctypes.POINTER(QsvmSvcProblem), _i32]),
    "qsvm_svc_fit": (_i32, [_dp, _i64, ctypes.POINTER(QsvmSvcProblem), _i32, ctypes.c_double, ctypes.c_double, _i64,
                            _dp, _vp, _vp, _sz, _vp]),
    "qsvm_svc_decision": (_i32, [_dp, _i64, _i64, ctypes.POINTER(QsvmSvcProblem), _i32, _dp, _dp, _vp, _sz, _vp]),
    "qsvm_sv_gram": (_i32, [_dp, _i64, _i32, _i32, _dp, _i64, _vp, _sz, _vp]),
    "qsvm_last_error": (ctypes.c_char_p, []),
    "qsvm_version": (ctypes.c_char_p, []),
}


def header_symbols() -> list[str]:
    """Function names declared in include/qsvm.h."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(qsvm_[a-z0-9_]+)\s*\(", text)))


def lib():
    """Load libqsvm.so (raises if it is missing: no fallback exists)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing; build it with paper_2405_02630_gb300.build")
            L = ctypes.CDLL(LIB_PATH)
            for name, (res, args) in _SIGS.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _check(rc: int):
    if rc != QSVM_OK:
        raise QsvmError(rc, lib().qsvm_last_error().decode())


def _prec(p) -> int:
    return PRECISIONS[p] if isinstance(p, str) else int(p)


def _stream(stream):
    import torch
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _optional_out(out, shape, **kw):
    """An optional float64 output argument: True allocates one, False or None means
    none, a tensor is used as given."""
    import torch
    if out is True:
        return torch.empty(shape, dtype=torch.float64, **kw)
    if out is False or out is None:
        return None
    return out


# ---------------------------------------------------------------- queries ---
def qsvm_mps_record_bytes(reps: int, precision) -> int:
    return int(lib().qsvm_mps_record_bytes(reps, _prec(precision)))


def qsvm_mps_point_bytes(n_qubits: int, reps: int, precision) -> int:
    return int(lib().qsvm_mps_point_bytes(n_qubits, reps, _prec(precision)))


def qsvm_mps_bytes(n_qubits: int, reps: int, n_points: int, precision) -> int:
    return int(lib().qsvm_mps_bytes(n_qubits, reps, n_points, _prec(precision)))


def qsvm_gram_tile_dim(reps: int, precision) -> int:
    return int(lib().qsvm_gram_tile_dim(reps, _prec(precision)))


def qsvm_gram_num_tiles(n_points: int, reps: int, precision) -> int:
    return int(lib().qsvm_gram_num_tiles(n_points, reps, _prec(precision)))


def qsvm_gram_partition(n_points: int, reps: int, precision, world: int, rank: int):
    b, e = _i64(0), _i64(0)
    _check(lib().qsvm_gram_partition(n_points, reps, _prec(precision), world, rank, ctypes.byref(b),
                                     ctypes.byref(e)))
    return int(b.value), int(e.value)


def qsvm_gram_tile_coords(n_points: int, reps: int, precision, tile: int):
    """(ti, tj) of Gram tile `tile` in the kernels' tile order."""
    a, b = _i64(0), _i64(0)
    _check(lib().qsvm_gram_tile_coords(n_points, reps, _prec(precision), tile, ctypes.byref(a), ctypes.byref(b)))
    return int(a.value), int(b.value)


def qsvm_gram_tile_list(n_points: int, reps: int, precision, tile_begin: int, tile_end: int):
    """(ti, tj) int64 numpy arrays of the Gram tiles [tile_begin, tile_end) in the kernels' order."""
    import numpy as np
    m = tile_end - tile_begin
    ti = np.empty(max(m, 0), dtype=np.int64)
    tj = np.empty(max(m, 0), dtype=np.int64)
    _check(lib().qsvm_gram_tile_list(n_points, reps, _prec(precision), tile_begin, tile_end,
                                     ti.ctypes.data if m > 0 else None, tj.ctypes.data if m > 0 else None))
    return ti, tj


# ---------------------------------------------------------------- compute ---
def qsvm_build_mps(X, reps: int, precision, mps=None, stream=None):
    """X: CUDA float64 (n_points, n_qubits), contiguous.  Returns the MPS buffer
    (a CUDA uint8 tensor of qsvm_mps_bytes bytes; allocated if not given)."""
    import torch
    assert X.is_cuda and X.dtype == torch.float64 and X.is_contiguous() and X.dim() == 2
    N, n = X.shape
    prec = _prec(precision)
    need = qsvm_mps_bytes(n, reps, N, prec)
    if mps is None:
        mps = torch.empty(max(need, 16), dtype=torch.uint8, device=X.device)
    _check(lib().qsvm_build_mps(_ptr(X), N, n, reps, prec, _ptr(mps), mps.numel() * mps.element_size(),
                                _stream(stream)))
    return mps


def qsvm_kernel_gram(mps, n_points: int, n_qubits: int, reps: int, precision, K=None, logK=False, stream=None,
                     device=None):
    """Symmetric Gram from an MPS buffer.  Returns (K, logK or None)."""
    import torch
    dev = device or mps.device
    if K is None:
        K = torch.empty((n_points, n_points), dtype=torch.float64, device=dev)
    L = _optional_out(logK, (n_points, n_points), device=dev)
    _check(lib().qsvm_kernel_gram(_ptr(mps), n_points, n_qubits, reps, _prec(precision), _ptr(K), K.stride(0),
                                  _ptr(L), L.stride(0) if L is not None else 0, _stream(stream)))
    return K, L


def qsvm_kernel_gram_tiles(mps, n_points: int, n_qubits: int, reps: int, precision, tile_begin: int, tile_end: int,
                           K, logK=None, stream=None):
    _check(lib().qsvm_kernel_gram_tiles(_ptr(mps), n_points, n_qubits, reps, _prec(precision), tile_begin, tile_end,
                                        _ptr(K), K.stride(0), _ptr(logK), logK.stride(0) if logK is not None else 0,
                                        _stream(stream)))
    return K, logK


def qsvm_kernel_cross(mps_a, n_a: int, mps_b, n_b: int, n_qubits: int, reps: int, precision, K=None, logK=False,
                      stream=None):
    """Test x train kernel: K[i, j] = |<psi(train_j)|psi(test_i)>|^2.  Returns (K, logK or None)."""
    import torch
    dev = mps_a.device
    if K is None:
        K = torch.empty((n_a, n_b), dtype=torch.float64, device=dev)
    L = _optional_out(logK, (n_a, n_b), device=dev)
    _check(lib().qsvm_kernel_cross(_ptr(mps_a), n_a, _ptr(mps_b), n_b, n_qubits, reps, _prec(precision), _ptr(K),
                                   K.stride(0), _ptr(L), L.stride(0) if L is not None else 0, _stream(stream)))
    return K, L


# ------------------------------------------------------------------ batch ---
def _jobs_array(jobs):
    """jobs: list of dicts with mps (uint8 tensor), n_points, n_qubits, K (tensor), logK (tensor or None)."""
    arr = (QsvmJob * len(jobs))()
    for k, j in enumerate(jobs):
        K, L = j["K"], j.get("logK")
        arr[k] = QsvmJob(j["mps"].data_ptr(), j["n_points"], j["n_qubits"], 0, K.data_ptr(), K.stride(0),
                         L.data_ptr() if L is not None else None, L.stride(0) if L is not None else 0)
    return arr


def qsvm_batch_workspace_bytes(n_jobs: int) -> int:
    return int(lib().qsvm_batch_workspace_bytes(n_jobs))


def qsvm_kernel_batch(jobs, reps: int, precision, ws, stream=None):
    arr = _jobs_array(jobs)
    _check(lib().qsvm_kernel_batch(arr, len(jobs), reps, _prec(precision), _ptr(ws), ws.numel() * ws.element_size(),
                                   _stream(stream)))


def qsvm_kernel_batch_noalloc(jobs, reps: int, precision, stream=None):
    """The batch without a workspace: for callers that must not allocate device
    memory; its scratch is a fixed array inside the library (at most 1024 jobs,
    calls must not overlap on the GPU)."""
    arr = _jobs_array(jobs)
    _check(lib().qsvm_kernel_batch_noalloc(arr, len(jobs), reps, _prec(precision), _stream(stream)))


class BatchPlan:
    """A CUDA-graph replay of one persistent multi-job launch (qsvm_batch_plan_*)."""

    def __init__(self, jobs, reps: int, precision, ws):
        self._keep = (jobs, ws)  # the plan uses these buffers until destroyed
        arr = _jobs_array(jobs)
        h = ctypes.c_void_p()
        _check(lib().qsvm_batch_plan_create(arr, len(jobs), reps, _prec(precision), _ptr(ws),
                                            ws.numel() * ws.element_size(), ctypes.byref(h)))
        self._h = h

    def launch(self, stream=None):
        _check(lib().qsvm_batch_plan_launch(self._h, _stream(stream)))

    def close(self):
        if self._h:
            lib().qsvm_batch_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def qsvm_batch_plan_create(jobs, reps: int, precision, ws) -> BatchPlan:
    return BatchPlan(jobs, reps, precision, ws)


# ---------------------------------------------------------------- configs ---
def qsvm_num_configs() -> int:
    return int(lib().qsvm_num_configs())


def qsvm_config_info(index: int, reps: int, precision):
    s, st = _i32(0), _i32(0)
    _check(lib().qsvm_config_info(index, reps, _prec(precision), ctypes.byref(s), ctypes.byref(st)))
    return int(s.value), int(st.value)


def qsvm_config_tile(index: int, reps: int, precision):
    """(pairs per side, threads per pair) of the block one CTA contracts under `index`."""
    a, b = _i32(), _i32()
    _check(lib().qsvm_config_tile(index, reps, _prec(precision), ctypes.byref(a), ctypes.byref(b)))
    return a.value, b.value


def qsvm_set_config(reps: int, precision, index: int):
    _check(lib().qsvm_set_config(reps, _prec(precision), index))


def qsvm_get_config(reps: int, precision) -> int:
    return int(lib().qsvm_get_config(reps, _prec(precision)))


def qsvm_autotune(mps, n_points: int, n_qubits: int, reps: int, precision, K, stream=None):
    """Times every configuration on this Gram, selects the fastest; returns (best, ms list)."""
    nc = qsvm_num_configs()
    ms = (ctypes.c_float * nc)()
    best = _i32(-1)
    _check(lib().qsvm_autotune(_ptr(mps), n_points, n_qubits, reps, _prec(precision), _ptr(K), K.stride(0),
                               _stream(stream), ctypes.byref(best), ms))
    return int(best.value), [float(v) for v in ms]


def qsvm_device_status(clear: bool = True, stream=None) -> int:
    v = _i32(0)
    _check(lib().qsvm_device_status(_stream(stream), 1 if clear else 0, ctypes.byref(v)))
    return int(v.value)


def qsvm_sv_workspace_bytes(n_points: int, n_qubits: int) -> int:
    return int(lib().qsvm_sv_workspace_bytes(n_points, n_qubits))


def qsvm_sv_gram(X, reps: int, K=None, ws=None, stream=None):
    """State-vector Gram (Algorithm 1 recipe on the GPU) of the rows of X (small n)."""
    import torch
    N, n = X.shape
    if K is None:
        K = torch.empty((N, N), dtype=torch.float64, device=X.device)
    if ws is None:
        ws = torch.empty(max(16, qsvm_sv_workspace_bytes(N, n)), dtype=torch.uint8, device=X.device)
    _check(lib().qsvm_sv_gram(_ptr(X), N, n, reps, _ptr(K), K.stride(0), _ptr(ws), ws.numel(), _stream(stream)))
    return K


# ------------------------------------------------------------------- SVC ---
def _svc_array(problems):
    """problems: list of dicts with idx (int64 tensor), y (int8 tensor), alpha (float64 tensor)."""
    arr = (QsvmSvcProblem * len(problems))()
    for k, p in enumerate(problems):
        arr[k] = QsvmSvcProblem(p["idx"].data_ptr(), p["y"].data_ptr(), p["idx"].numel(), p["alpha"].data_ptr())
    return arr


def qsvm_svc_workspace_bytes(problems) -> int:
    arr = _svc_array(problems)
    return int(lib().qsvm_svc_workspace_bytes(arr, len(problems)))


def qsvm_svc_fit(K, problems, C: float = 1.0, tol: float = 1e-8, max_iter: int = 10_000_000, stream=None):
    """SMO on each binary problem (one CTA each).  Returns (b, iters) device tensors."""
    import torch
    arr = _svc_array(problems)
    ws = torch.empty(max(256, int(lib().qsvm_svc_workspace_bytes(arr, len(problems)))), dtype=torch.uint8,
                     device=K.device)
    b = torch.empty(len(problems), dtype=torch.float64, device=K.device)
    it = torch.empty(len(problems), dtype=torch.int64, device=K.device)
    _check(lib().qsvm_svc_fit(_ptr(K), K.stride(0), arr, len(problems), C, tol, max_iter, _ptr(b), _ptr(it), _ptr(ws),
                              ws.numel(), _stream(stream)))
    return b, it


def qsvm_svc_decision(Kx, problems, b, stream=None):
    """F[r, p] = sum_i alpha_i y_i Kx[r, idx_i] + b[p]."""
    import torch
    arr = _svc_array(problems)
    ws = torch.empty(max(256, 256 * ((len(problems) * 40 + 255) // 256)), dtype=torch.uint8, device=Kx.device)
    F = torch.empty((Kx.shape[0], len(problems)), dtype=torch.float64, device=Kx.device)
    _check(lib().qsvm_svc_decision(_ptr(Kx), Kx.stride(0), Kx.shape[0], arr, len(problems), _ptr(b), _ptr(F),
                                   _ptr(ws), ws.numel(), _stream(stream)))
    return F


def qsvm_selftest_wait_timeout(limit_ns: int, stream=None):
    _check(lib().qsvm_selftest_wait_timeout(limit_ns, _stream(stream)))


def qsvm_last_error() -> str:
    return lib().qsvm_last_error().decode()


def qsvm_version() -> str:
    return lib().qsvm_version().decode()


# ------------------------------------------------------------ convenience ---
def qsvm_gram_host_workspace_bytes(n_points: int, n_qubits: int, reps: int, precision, with_logk: bool = False) -> int:
    return int(lib().qsvm_gram_host_workspace_bytes(n_points, n_qubits, reps, _prec(precision), int(bool(with_logk))))


def gram_host(X, reps: int, precision, K=None, logK=True, ws=None, stream=None):
    """The Gram of host data through qsvm_gram_host.  X: contiguous CPU float64 tensor
    (page-locked for asynchronous copies); K, logK: CPU float64 outputs (page-locked ones
    are allocated if not given; logK=False skips ln K); ws: device scratch (allocated if
    not given).  Returns (K, logK or None), complete once `stream` (default: the current
    stream) is synchronised.  ln K is returned by default: at hundreds of qubits almost
    every off-diagonal K underflows to 0 in FP64 while ln K stays exact."""
    import torch
    if X.device.type != "cpu" or X.dtype != torch.float64 or not X.is_contiguous():
        raise ValueError("X must be a contiguous CPU float64 tensor")
    N, n = X.shape
    if K is None:
        K = torch.empty((N, N), dtype=torch.float64, pin_memory=True)
    L = _optional_out(logK, (N, N), pin_memory=True)
    need = qsvm_gram_host_workspace_bytes(N, n, reps, precision, L is not None)
    if ws is None:
        ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    _check(lib().qsvm_gram_host(_ptr(X), N, n, reps, _prec(precision), _ptr(K), K.stride(0), _ptr(L),
                                L.stride(0) if L is not None else 0, _ptr(ws), ws.numel(), _stream(stream)))
    return K, L


def qsvm_cross_host_workspace_bytes(n_a: int, n_b: int, n_qubits: int, reps: int, precision,
                                    with_logk: bool = False) -> int:
    return int(lib().qsvm_cross_host_workspace_bytes(n_a, n_b, n_qubits, reps, _prec(precision), int(bool(with_logk))))


def cross_host(X_test, X_train, reps: int, precision, K=None, logK=True, ws=None, stream=None):
    """Test x train kernel of host data through qsvm_cross_host (contiguous CPU float64
    inputs; page-locked outputs allocated if not given; ln K unless logK=False).  Returns
    (K, logK or None), complete once `stream` is synchronised."""
    import torch
    for X in (X_test, X_train):
        if X.device.type != "cpu" or X.dtype != torch.float64 or not X.is_contiguous():
            raise ValueError("X_test and X_train must be contiguous CPU float64 tensors")
    na, n = X_test.shape
    nb = X_train.shape[0]
    if K is None:
        K = torch.empty((na, nb), dtype=torch.float64, pin_memory=True)
    L = _optional_out(logK, (na, nb), pin_memory=True)
    need = qsvm_cross_host_workspace_bytes(na, nb, n, reps, precision, L is not None)
    if ws is None:
        ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    _check(lib().qsvm_cross_host(_ptr(X_test), na, _ptr(X_train), nb, n, reps, _prec(precision), _ptr(K), K.stride(0),
                                 _ptr(L), L.stride(0) if L is not None else 0, _ptr(ws), ws.numel(), _stream(stream)))
    return K, L


def gram(X, reps: int, precision, logK: bool = True, stream=None):
    """Build the MPS of every row of X and return its Gram (K, logK), or (K, None) with
    logK=False.  ln K is the default output: at hundreds of qubits K itself underflows
    to 0 off the diagonal (kernel concentration) while ln K keeps the information."""
    N, n = X.shape
    mps = qsvm_build_mps(X, reps, precision, stream=stream)
    return qsvm_kernel_gram(mps, N, n, reps, precision, logK=logK, stream=stream)


def cross(X_test, X_train, reps: int, precision, logK: bool = True, stream=None):
    """Test x train kernel of two feature matrices (K, logK), or (K, None) with logK=False."""
    ma = qsvm_build_mps(X_test, reps, precision, stream=stream)
    mb = qsvm_build_mps(X_train, reps, precision, stream=stream)
    return qsvm_kernel_cross(ma, X_test.shape[0], mb, X_train.shape[0], X_test.shape[1], reps, precision, logK=logK,
                             stream=stream)
