"""Batched persistent launch, its CUDA-graph plan and the autotuner, on the GPU.

Every pipeline configuration and the persistent kernel run the same arithmetic
in the same order, so their results must be bit-identical to the per-tile Gram;
against the oracle the usual tolerances apply.
"""
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


def _jobs(q, specs, reps, prec, seed, logk=True):
    rng = np.random.default_rng(seed)
    jobs, Xs = [], []
    for N, n in specs:
        X = rng.random((N, n)) * np.pi
        Xd = torch.from_numpy(X).cuda()
        mps = q.qsvm_build_mps(Xd, reps, prec)
        K = torch.full((N, N), float("nan"), dtype=torch.float64, device="cuda")
        L = torch.full((N, N), float("nan"), dtype=torch.float64, device="cuda") if logk else None
        jobs.append({"mps": mps, "n_points": N, "n_qubits": n, "K": K, "logK": L})
        Xs.append(X)
    return jobs, Xs


SPECS = [(37, 16), (80, 64), (17, 130), (64, 16), (5, 64), (33, 40)]


# every compiled persistent kernel: chi = 2, 4, 8 (reps 1, 2, 3) in each precision
@pytest.mark.parametrize("prec,reps", [("fp64", 2), ("fp32_split", 2), ("fp32", 2), ("fp32_split", 3), ("fp64", 3),
                                       ("fp32", 3), ("fp64", 1), ("fp32_split", 1), ("fp32", 1)])
def test_batch_matches_per_job_gram(q, oracle, prec, reps):
    jobs, Xs = _jobs(q, SPECS, reps, prec, 1)
    ws = torch.empty(q.qsvm_batch_workspace_bytes(len(jobs)), dtype=torch.uint8, device="cuda")
    q.qsvm_kernel_batch(jobs, reps, prec, ws)
    torch.cuda.synchronize()
    assert q.qsvm_device_status() == 0
    tol = {"fp64": 1e-10, "fp32_split": 1e-6, "fp32": 2e-5}[prec]
    for j, X in zip(jobs, Xs):
        Kref, Lref = q.qsvm_kernel_gram(j["mps"], j["n_points"], j["n_qubits"], reps, prec, logK=True)
        assert torch.equal(j["K"], Kref) and torch.equal(j["logK"], Lref)
        Ko, _ = oracle.mps_gram(X, reps)
        assert np.max(np.abs(j["K"].cpu().numpy() - Ko)) <= tol


def test_batch_plan_replays(q):
    reps, prec = 2, "fp32_split"
    jobs, _ = _jobs(q, SPECS, reps, prec, 2, logk=False)
    ws = torch.empty(q.qsvm_batch_workspace_bytes(len(jobs)), dtype=torch.uint8, device="cuda")
    plan = q.qsvm_batch_plan_create(jobs, reps, prec, ws)
    plan.launch()
    torch.cuda.synchronize()
    first = [j["K"].clone() for j in jobs]
    for j in jobs:
        j["K"].fill_(float("nan"))
    plan.launch()
    plan.launch()
    torch.cuda.synchronize()
    for j, K0 in zip(jobs, first):
        assert torch.equal(j["K"], K0)
        Kref, _ = q.qsvm_kernel_gram(j["mps"], j["n_points"], j["n_qubits"], reps, prec)
        assert torch.equal(K0, Kref)
    plan.close()


@pytest.mark.parametrize("reps", [1, 2, 3])
def test_every_config_bit_identical(q, reps):
    prec = "fp32_split"
    N, n = 40, 50
    X = torch.from_numpy(inputs.uniform_features(N, n, 3)).cuda()
    mps = q.qsvm_build_mps(X, reps, prec)
    q.qsvm_set_config(reps, prec, -1)
    Kdef, _ = q.qsvm_kernel_gram(mps, N, n, reps, prec)
    ran = 0
    for c in range(q.qsvm_num_configs()):
        try:
            q.qsvm_set_config(reps, prec, c)
        except q.QsvmError as e:  # the shape needs more shared memory than a CTA has
            assert e.code == q.QSVM_ERR_ARG
            continue
        Kc, _ = q.qsvm_kernel_gram(mps, N, n, reps, prec)
        assert torch.equal(Kc, Kdef), c
        ran += 1
    assert ran >= 2
    q.qsvm_set_config(reps, prec, -1)


@pytest.mark.parametrize("prec", ["fp64", "fp32_split", "fp32"])
@pytest.mark.parametrize("reps", [1, 2, 3])
@pytest.mark.parametrize("N,Nt", [(37, 21), (1, 1), (9, 5)])
def test_quarter_tile_configs_vs_oracle(q, oracle, prec, reps, N, Nt):
    """Configurations that give each CTA a quarter of a tile: Gram and cross kernel with
    ragged edges (quarters beyond the last row or column, the skipped quarter below a
    diagonal tile; a single point) against the oracle, and bit-identical to the
    whole-tile default."""
    tol = {"fp64": 1e-10, "fp32_split": 1e-6, "fp32": 2e-5}[prec]
    n = 13
    X, Xt = inputs.uniform_features(N, n, 61), inputs.uniform_features(Nt, n, 62)
    Ko, _ = oracle.mps_gram(X, reps)
    Kxo, _ = oracle.mps_cross(Xt, X, reps)
    Xd, Xtd = torch.from_numpy(X).cuda(), torch.from_numpy(Xt).cuda()
    q.qsvm_set_config(reps, prec, -1)
    Kdef, Ldef = q.gram(Xd, reps, prec)
    Kxdef, _ = q.cross(Xtd, Xd, reps, prec)
    half = q.qsvm_num_configs() // 2
    try:
        for c in (half + 3, half + 9):
            q.qsvm_set_config(reps, prec, c)
            side, _ = q.qsvm_config_tile(c, reps, prec)
            assert side == q.qsvm_gram_tile_dim(reps, prec) // 2
            K, L = q.gram(Xd, reps, prec)
            Kx, _ = q.cross(Xtd, Xd, reps, prec)
            torch.cuda.synchronize()
            assert q.qsvm_device_status() == 0
            assert torch.equal(K, Kdef) and torch.equal(L, Ldef) and torch.equal(Kx, Kxdef)
            assert float(np.max(np.abs(K.cpu().numpy() - Ko))) <= tol
            assert float(np.max(np.abs(Kx.cpu().numpy() - Kxo))) <= tol
    finally:
        q.qsvm_set_config(reps, prec, -1)


def test_autotune_selects_a_config(q, tmp_path, monkeypatch):
    from paper_2405_02630_gb300 import autotune
    monkeypatch.setenv("QSVM_AUTOTUNE_CACHE", str(tmp_path / "at.json"))
    reps, prec = 2, "fp32_split"
    N, n = 96, 200
    X = torch.from_numpy(inputs.mnist_like_features(N, n, 5)).cuda()
    mps = q.qsvm_build_mps(X, reps, prec)
    K = torch.empty((N, N), dtype=torch.float64, device="cuda")
    rec = autotune.tune(mps, N, n, reps, prec, K)
    assert 0 <= rec["config"] < q.qsvm_num_configs()
    assert q.qsvm_get_config(reps, prec) == rec["config"]
    assert min(m for m in rec["ms"] if m > 0) == rec["ms"][rec["config"]]
    q.qsvm_set_config(reps, prec, -1)
    assert autotune.apply_cached(reps, prec, n) == rec["config"]
    q.qsvm_set_config(reps, prec, -1)
