"""The C-ABI library loads, exports every symbol include/qsvm.h declares, and its
pure-host logic (argument checks, sizes, tile partition) behaves -- no GPU needed:
every call here returns before touching CUDA."""
import ctypes

import pytest

from paper_2405_02630_gb300 import qsvm


def test_exports_every_declared_symbol():
    L = qsvm.lib()
    names = qsvm.header_symbols()
    assert len(names) >= 12
    for name in names:
        assert hasattr(L, name), name
    assert set(names) == set(qsvm._SIGS), "binding and header disagree"


def test_record_and_mps_bytes():
    # block form (reps 1, 3): per site the blocks a_00, a_01 (chi^2 / 2 complex entries) and
    # the phase r, 16 bytes each; split FP32 holds hi and lo; FP32 formats hold two forms
    for reps, chi in ((1, 2), (3, 8)):
        entries = 2 * (chi // 2) ** 2 + 1  # blocks a_00, a_01 and the phase r
        assert qsvm.qsvm_mps_record_bytes(reps, "fp32") == entries * 16
    assert qsvm.qsvm_mps_record_bytes(1, "fp64") == 3 * 16
    # FP64 at reps = 3: the gauged records of reps = 2 (alpha, beta doubles, n + 1 per point)
    assert qsvm.qsvm_mps_record_bytes(3, "fp64") == 32
    assert qsvm.qsvm_mps_bytes(64, 3, 10, "fp64") == 10 * 65 * 32
    assert qsvm.qsvm_mps_record_bytes(1, "fp32_split") == 3 * 32
    assert qsvm.qsvm_mps_bytes(64, 3, 10, "fp32") == 2 * 10 * 64 * 33 * 16
    # split FP32 at reps = 3: the gauged records of reps = 2 (alpha, beta; hi, lo; two arrays of
    # n + 1 records per point)
    assert qsvm.qsvm_mps_record_bytes(3, "fp32_split") == 64
    assert qsvm.qsvm_mps_bytes(64, 3, 10, "fp32_split") == 2 * 10 * 65 * 64
    # reps = 2: plain FP32 in phase form (three phases, both forms of 16 bytes); FP64 in gauged
    # form (alpha, beta doubles, n + 1 records per point, one array)
    assert qsvm.qsvm_mps_record_bytes(2, "fp64") == 32
    assert qsvm.qsvm_mps_record_bytes(2, "fp32") == 96
    assert qsvm.qsvm_mps_bytes(784, 2, 8192, "fp64") == 8192 * 785 * 32
    assert qsvm.qsvm_mps_bytes(784, 2, 8192, "fp32") == 8192 * 784 * 96
    # reps = 2, split FP32, gauged form: alpha and beta, hi and lo, per form; n + 1 records
    # (one virtual site) per point in a row-side and a column-side array
    assert qsvm.qsvm_mps_record_bytes(2, "fp32_split") == 64
    assert qsvm.qsvm_mps_point_bytes(784, 2, "fp32_split") == 785 * 64
    assert qsvm.qsvm_mps_bytes(784, 2, 8192, "fp32_split") == 2 * 8192 * 785 * 64
    # the row stride of one array: sites x record bytes (block form: two arrays)
    assert qsvm.qsvm_mps_point_bytes(784, 2, "fp64") == 785 * 32
    assert qsvm.qsvm_mps_point_bytes(64, 3, "fp32") == 64 * 33 * 16
    assert qsvm.qsvm_mps_point_bytes(64, 3, "fp32_split") == 65 * 64
    assert qsvm.qsvm_mps_point_bytes(0, 2, "fp64") == 0 and qsvm.qsvm_mps_point_bytes(8, 4, "fp64") == 0
    assert qsvm.qsvm_mps_record_bytes(4, "fp64") == 0
    assert qsvm.qsvm_mps_record_bytes(2, 7) == 0


def _call_gram(**kw):
    a = dict(mps=16, n=16, nq=8, reps=2, prec=0, K=64, ldk=16, L=None, ldl=0)
    a.update(kw)
    return qsvm.lib().qsvm_kernel_gram(ctypes.c_void_p(a["mps"]), a["n"], a["nq"], a["reps"], a["prec"],
                                       ctypes.c_void_p(a["K"]), a["ldk"], ctypes.c_void_p(a["L"]) if a["L"] else None,
                                       a["ldl"], None)


@pytest.mark.parametrize("kw,code", [
    (dict(reps=0), qsvm.QSVM_ERR_CHI), (dict(reps=4), qsvm.QSVM_ERR_CHI), (dict(nq=1), qsvm.QSVM_ERR_ARG),
    (dict(prec=3), qsvm.QSVM_ERR_ARG), (dict(n=0), qsvm.QSVM_ERR_ARG), (dict(mps=0), qsvm.QSVM_ERR_ARG),
    (dict(mps=8), qsvm.QSVM_ERR_ARG), (dict(K=0), qsvm.QSVM_ERR_ARG), (dict(ldk=15), qsvm.QSVM_ERR_ARG),
    (dict(L=64, ldl=3), qsvm.QSVM_ERR_ARG),
])
def test_gram_argument_errors(kw, code):
    assert _call_gram(**kw) == code
    assert qsvm.qsvm_last_error()


def test_build_and_cross_argument_errors():
    L = qsvm.lib()
    v = ctypes.c_void_p
    assert L.qsvm_build_mps(v(64), 4, 8, 2, 0, v(64), 10, None) == qsvm.QSVM_ERR_ARG  # mps_bytes too small
    assert L.qsvm_build_mps(None, 4, 8, 2, 0, v(64), 1 << 20, None) == qsvm.QSVM_ERR_ARG
    assert L.qsvm_build_mps(v(64), 4, 8, 5, 0, v(64), 1 << 20, None) == qsvm.QSVM_ERR_CHI
    assert L.qsvm_kernel_cross(v(16), 4, v(16), 0, 8, 2, 0, v(64), 4, None, 0, None) == qsvm.QSVM_ERR_ARG
    assert L.qsvm_kernel_cross(v(16), 4, v(16), 5, 8, 2, 0, v(64), 4, None, 0, None) == qsvm.QSVM_ERR_ARG
    assert L.qsvm_kernel_gram_tiles(v(16), 16, 8, 2, 0, 0, 99, v(64), 16, None, 0, None) == qsvm.QSVM_ERR_ARG


def _tile_pairs(b, N, T, td):
    ti, tj = qsvm.qsvm_gram_tile_coords(N, 2, "fp32_split", b)
    ni, nj = min(td, N - ti * td), min(td, N - tj * td)
    return ni * (ni + 1) // 2 if ti == tj else ni * nj


@pytest.mark.parametrize("N", [1, 16, 17, 100, 129, 1000, 2049, 4100])
def test_tile_order_covers_upper_triangle_once(N):
    td = qsvm.qsvm_gram_tile_dim(2, "fp32_split")
    T = -(-N // td)
    total = qsvm.qsvm_gram_num_tiles(N, 2, "fp32_split")
    seen = [qsvm.qsvm_gram_tile_coords(N, 2, "fp32_split", b) for b in range(total)]
    assert len(set(seen)) == total == T * (T + 1) // 2
    assert all(0 <= ti <= tj < T for ti, tj in seen)
    # bands of 64 tile rows, visited in order
    bands = [ti // 64 for ti, _ in seen]
    assert bands == sorted(bands)
    with pytest.raises(qsvm.QsvmError):
        qsvm.qsvm_gram_tile_coords(N, 2, "fp32_split", total)


@pytest.mark.parametrize("N,world", [(1, 1), (17, 2), (100, 3), (1000, 8), (8192, 4), (33, 7)])
def test_gram_partition_covers_and_balances(N, world):
    td = qsvm.qsvm_gram_tile_dim(2, "fp32_split")
    T = -(-N // td)
    total = qsvm.qsvm_gram_num_tiles(N, 2, "fp32_split")
    assert total == T * (T + 1) // 2
    ranges = [qsvm.qsvm_gram_partition(N, 2, "fp32_split", world, r) for r in range(world)]
    assert ranges[0][0] == 0 and ranges[-1][1] == total
    assert all(ranges[r][1] == ranges[r + 1][0] for r in range(world - 1))
    pairs = [sum(_tile_pairs(b, N, T, td) for b in range(lo, hi)) for lo, hi in ranges]
    assert sum(pairs) == N * (N + 1) // 2
    if total >= 4 * world:
        assert max(pairs) - min(pairs) <= 2 * td * td


def test_partition_errors():
    with pytest.raises(qsvm.QsvmError):
        qsvm.qsvm_gram_partition(100, 2, 0, 2, 2)
    with pytest.raises(qsvm.QsvmError):
        qsvm.qsvm_gram_partition(0, 2, 0, 1, 0)


def test_batch_workspace_and_argument_errors():
    assert qsvm.qsvm_batch_workspace_bytes(0) == 0
    w1, w32 = qsvm.qsvm_batch_workspace_bytes(1), qsvm.qsvm_batch_workspace_bytes(32)
    assert w1 % 256 == 0 and w32 % 256 == 0 and w32 >= 256 + 64 * 32 + 8 * 33
    L = qsvm.lib()
    job = qsvm.QsvmJob(256, 10, 8, 0, 512, 10, None, 0)
    arr = (qsvm.QsvmJob * 1)(job)
    v = ctypes.c_void_p
    assert L.qsvm_kernel_batch(None, 1, 2, 2, v(4096), 1 << 20, None) == qsvm.QSVM_ERR_ARG
    assert L.qsvm_kernel_batch(arr, 1, 2, 2, v(4096), 16, None) == qsvm.QSVM_ERR_WORKSPACE
    assert L.qsvm_kernel_batch(arr, 1, 2, 2, v(4100), 1 << 20, None) == qsvm.QSVM_ERR_ARG  # misaligned ws
    assert L.qsvm_kernel_batch(arr, 1, 4, 2, v(4096), 1 << 20, None) == qsvm.QSVM_ERR_CHI
    bad = (qsvm.QsvmJob * 1)(qsvm.QsvmJob(256, 10, 8, 0, 512, 9, None, 0))  # ldk < n_points
    assert L.qsvm_kernel_batch(bad, 1, 2, 2, v(4096), 1 << 20, None) == qsvm.QSVM_ERR_ARG
    h = ctypes.c_void_p()
    assert L.qsvm_batch_plan_create(bad, 1, 2, 2, v(4096), 1 << 20, ctypes.byref(h)) == qsvm.QSVM_ERR_ARG
    assert L.qsvm_batch_plan_launch(None, None) == qsvm.QSVM_ERR_ARG
    assert L.qsvm_batch_plan_destroy(None) == qsvm.QSVM_OK


def test_configs():
    n = qsvm.qsvm_num_configs()
    assert n >= 4
    for reps in (1, 2, 3):
        for prec in ("fp64", "fp32", "fp32_split"):
            for c in range(n):
                S, st = qsvm.qsvm_config_info(c, reps, prec)
                assert S >= 1 and 2 <= st <= 4
    S2, _ = qsvm.qsvm_config_info(1, 2, "fp32_split")
    assert S2 == 16  # 1 KB of 64-byte records per point and chunk
    # the first half of the configurations give a CTA a whole tile, the second half a quarter
    for reps, prec, side, tpp in ((1, "fp64", 16, 1), (2, "fp32_split", 16, 1), (3, "fp32_split", 8, 4),
                                  (3, "fp64", 16, 1)):
        assert qsvm.qsvm_gram_tile_dim(reps, prec) == side
        assert qsvm.qsvm_config_tile(-1, reps, prec) == (side, tpp)
        for c in range(n):
            assert qsvm.qsvm_config_tile(c, reps, prec) == (side if c < n // 2 else side // 2, tpp)
            assert qsvm.qsvm_config_info(c, reps, prec) == qsvm.qsvm_config_info(c % (n // 2), reps, prec)
    with pytest.raises(qsvm.QsvmError):
        qsvm.qsvm_config_tile(n, 2, "fp32_split")
    assert qsvm.qsvm_get_config(2, "fp64") == -1
    qsvm.qsvm_set_config(2, "fp64", 0)
    assert qsvm.qsvm_get_config(2, "fp64") == 0
    qsvm.qsvm_set_config(2, "fp64", -1)
    with pytest.raises(qsvm.QsvmError):
        qsvm.qsvm_set_config(2, "fp64", n)


def test_autotune_buckets():
    from paper_2405_02630_gb300 import autotune
    assert [autotune.n_bucket(n) for n in (2, 16, 17, 784)] == [2, 16, 32, 1024]


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(qsvm, "LIB_PATH", str(tmp_path / "missing" / "libqsvm.so"))
    monkeypatch.setattr(qsvm, "_lib", None)
    with pytest.raises(RuntimeError, match="missing"):
        qsvm.lib()
    with pytest.raises(RuntimeError):
        qsvm.qsvm_mps_bytes(8, 2, 4, "fp64")


def test_statevector_sizes_and_errors():
    assert qsvm.qsvm_sv_workspace_bytes(10, 8) == 10 * 256 * 16
    assert qsvm.qsvm_sv_workspace_bytes(10, 25) == 0
    L = qsvm.lib()
    v = ctypes.c_void_p
    assert L.qsvm_sv_gram(v(64), 4, 25, 2, v(64), 4, v(64), 1 << 30, None) == qsvm.QSVM_ERR_ARG
    assert L.qsvm_sv_gram(v(64), 4, 8, 0, v(64), 4, v(64), 1 << 30, None) == qsvm.QSVM_ERR_ARG
    assert L.qsvm_sv_gram(v(64), 4, 8, 2, v(64), 3, v(64), 1 << 30, None) == qsvm.QSVM_ERR_ARG
    assert L.qsvm_sv_gram(v(64), 4, 8, 2, v(64), 4, v(64), 100, None) == qsvm.QSVM_ERR_WORKSPACE


def test_weak_scaling_workload_sizes():
    """The bench's G-rank run grows the Gram to round(N sqrt(G)) points, so every rank's
    pair-balanced share stays near the one-GPU Gram's pair count."""
    from paper_2405_02630_gb300 import inputs
    N = inputs.WORKLOADS["gram_n784_r2_N8192"][2]
    for G in (1, 2, 4, 8):
        Ng = int(round(N * G ** 0.5))
        X, Xte, n, reps = inputs.workload("cfg0_n8_r2_N16", scale=G ** 0.5)
        assert X.shape == (int(round(16 * G ** 0.5)), 8) and Xte is None
        total = qsvm.qsvm_gram_num_tiles(Ng, reps, "fp32_split")
        shares = [qsvm.qsvm_gram_partition(Ng, reps, "fp32_split", G, r) for r in range(G)]
        assert shares[0][0] == 0 and shares[-1][1] == total
        per_rank_pairs = Ng * (Ng + 1) / 2 / G
        assert abs(per_rank_pairs / (N * (N + 1) / 2) - 1) < 1e-3


def test_gram_host_arguments():
    """qsvm_gram_host checks its arguments on the host before any copy or launch."""
    import ctypes
    L = qsvm.lib()
    v = lambda n: ctypes.c_void_p(256 * n)
    N, n = 100, 24
    need = qsvm.qsvm_gram_host_workspace_bytes(N, n, 2, "fp32_split")
    a256 = lambda b: (b + 255) // 256 * 256
    assert need == a256(N * n * 8) + a256(qsvm.qsvm_mps_bytes(n, 2, N, "fp32_split")) + a256(N * N * 8)
    assert qsvm.qsvm_gram_host_workspace_bytes(N, n, 2, "fp32_split", True) == need + a256(N * N * 8)
    assert qsvm.qsvm_gram_host_workspace_bytes(0, n, 2, "fp64") == 0
    assert qsvm.qsvm_gram_host_workspace_bytes(N, n, 4, "fp64") == 0
    ok = dict(X=v(1), N=N, n=n, reps=2, prec=2, K=v(2), ldk=N, lg=None, ldl=0, ws=v(3), wsb=need)
    def call(**kw):
        a = dict(ok); a.update(kw)
        return L.qsvm_gram_host(a["X"], a["N"], a["n"], a["reps"], a["prec"], a["K"], a["ldk"], a["lg"], a["ldl"],
                                a["ws"], a["wsb"], None)
    assert call(X=None) == qsvm.QSVM_ERR_ARG
    assert call(K=None) == qsvm.QSVM_ERR_ARG
    assert call(ldk=N - 1) == qsvm.QSVM_ERR_ARG
    assert call(lg=v(4), ldl=N - 1) == qsvm.QSVM_ERR_ARG
    assert call(lg=v(4), ldl=N) == qsvm.QSVM_ERR_ARG  # ws sized without logK
    assert call(ws=None) == qsvm.QSVM_ERR_ARG
    assert call(ws=ctypes.c_void_p(256 * 3 + 16)) == qsvm.QSVM_ERR_ARG  # misaligned
    assert call(wsb=need - 1) == qsvm.QSVM_ERR_ARG
    assert call(N=0) == qsvm.QSVM_ERR_ARG
    assert call(reps=4) == qsvm.QSVM_ERR_CHI


def test_cross_host_arguments():
    """qsvm_cross_host checks its arguments on the host before any copy or launch."""
    import ctypes
    L = qsvm.lib()
    v = lambda n: ctypes.c_void_p(256 * n)
    Na, Nb, n = 40, 100, 24
    a256 = lambda b: (b + 255) // 256 * 256
    need = qsvm.qsvm_cross_host_workspace_bytes(Na, Nb, n, 2, "fp32_split")
    assert need == (a256((Na + Nb) * n * 8) + a256(qsvm.qsvm_mps_bytes(n, 2, Na, "fp32_split"))
                    + a256(qsvm.qsvm_mps_bytes(n, 2, Nb, "fp32_split")) + a256(Na * Nb * 8))
    assert qsvm.qsvm_cross_host_workspace_bytes(Na, Nb, n, 2, "fp32_split", True) == need + a256(Na * Nb * 8)
    assert qsvm.qsvm_cross_host_workspace_bytes(0, Nb, n, 2, "fp64") == 0
    assert qsvm.qsvm_cross_host_workspace_bytes(Na, 0, n, 2, "fp64") == 0
    assert qsvm.qsvm_cross_host_workspace_bytes(Na, Nb, n, 4, "fp64") == 0
    ok = dict(Xa=v(1), Na=Na, Xb=v(5), Nb=Nb, n=n, reps=2, prec=2, K=v(2), ldk=Nb, lg=None, ldl=0, ws=v(3), wsb=need)
    def call(**kw):
        a = dict(ok); a.update(kw)
        return L.qsvm_cross_host(a["Xa"], a["Na"], a["Xb"], a["Nb"], a["n"], a["reps"], a["prec"], a["K"], a["ldk"],
                                 a["lg"], a["ldl"], a["ws"], a["wsb"], None)
    assert call(Xa=None) == qsvm.QSVM_ERR_ARG
    assert call(Xb=None) == qsvm.QSVM_ERR_ARG
    assert call(K=None) == qsvm.QSVM_ERR_ARG
    assert call(ldk=Nb - 1) == qsvm.QSVM_ERR_ARG
    assert call(lg=v(4), ldl=Nb - 1) == qsvm.QSVM_ERR_ARG
    assert call(lg=v(4), ldl=Nb) == qsvm.QSVM_ERR_ARG  # ws sized without logK
    assert call(ws=None) == qsvm.QSVM_ERR_ARG
    assert call(ws=ctypes.c_void_p(256 * 3 + 16)) == qsvm.QSVM_ERR_ARG  # misaligned
    assert call(wsb=need - 1) == qsvm.QSVM_ERR_ARG
    assert call(Na=0) == qsvm.QSVM_ERR_ARG
    assert call(Nb=0) == qsvm.QSVM_ERR_ARG
    assert call(reps=4) == qsvm.QSVM_ERR_CHI


def test_gram_tile_list():
    """qsvm_gram_tile_list decodes a tile range into host arrays (the kernels' order:
    equal to qsvm_gram_tile_coords tile by tile), an empty range needs no arrays, and a
    range outside [0, tiles] is an argument error."""
    import ctypes
    N, reps, prec = 300, 2, "fp32_split"
    total = qsvm.qsvm_gram_num_tiles(N, reps, prec)
    ti, tj = qsvm.qsvm_gram_tile_list(N, reps, prec, 5, total - 3)
    assert len(ti) == total - 8
    assert list(zip(ti, tj)) == [qsvm.qsvm_gram_tile_coords(N, reps, prec, b) for b in range(5, total - 3)]
    assert len(qsvm.qsvm_gram_tile_list(N, reps, prec, 7, 7)[0]) == 0
    L = qsvm.lib()
    buf = (ctypes.c_int64 * 4)()
    p = ctypes.cast(buf, ctypes.c_void_p)
    assert L.qsvm_gram_tile_list(N, reps, 2, -1, 2, p, p) == qsvm.QSVM_ERR_ARG
    assert L.qsvm_gram_tile_list(N, reps, 2, 3, 2, p, p) == qsvm.QSVM_ERR_ARG
    assert L.qsvm_gram_tile_list(N, reps, 2, total - 1, total + 1, p, p) == qsvm.QSVM_ERR_ARG
    assert L.qsvm_gram_tile_list(N, reps, 2, 0, 2, None, None) == qsvm.QSVM_ERR_ARG
    assert L.qsvm_gram_tile_list(0, reps, 2, 0, 0, None, None) == qsvm.QSVM_ERR_ARG
    # the union of every rank's range covers each tile once, in order
    from paper_2405_02630_gb300 import shard
    allt = [t for r in range(5) for t in zip(*shard.rank_tiles(N, reps, prec, 5, r))]
    assert allt == list(zip(*qsvm.qsvm_gram_tile_list(N, reps, prec, 0, total)))
