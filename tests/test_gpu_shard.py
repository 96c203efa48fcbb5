"""The sharded Gram on the GPU (the paper distributes pairs over GPUs and gathers K,
Sec. 5).  Every rank's tile range is computed by qsvm_kernel_gram_tiles into its own
NaN-filled buffer, packed and assembled as shard.gather_gram does (the exchange itself
is covered by the gloo tests; one GPU runs no collective between ranks).  The assembled
Gram must equal the single-call Gram bit-exactly and the CPU oracle element by element
at the precision's tolerance; shard.gram_sharded over a one-rank NCCL group must equal
qsvm.gram and the oracle."""
import socket

import numpy as np
import pytest
import torch

from paper_2405_02630_gb300 import inputs

pytestmark = pytest.mark.gpu

TOL = {"fp64": 1e-10, "fp32_split": 1e-6, "fp32": 2e-5}
LOG_TOL = {"fp64": 1e-8, "fp32_split": 1e-5, "fp32": 1e-3}


@pytest.fixture(scope="module")
def q():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2405_02630_gb300 import qsvm
    qsvm.lib()
    return qsvm


def _vs_oracle(K, L, Ko, LKo, prec, what):
    K, L = K.cpu().numpy(), L.cpu().numpy()
    err = np.max(np.abs(K - Ko))
    assert err <= TOL[prec], f"{what} {prec}: max|dK| = {err:.3e}"
    m = Ko > 1e-300
    lerr = np.max(np.abs(L[m] - LKo[m]))
    assert lerr <= LOG_TOL[prec], f"{what} {prec}: max|dlnK| = {lerr:.3e}"


@pytest.mark.parametrize("prec", ["fp64", "fp32_split", "fp32"])
@pytest.mark.parametrize("N,n,reps,world", [(300, 24, 2, 3), (77, 10, 1, 5), (200, 9, 3, 2), (20, 6, 2, 3)])
def test_rank_ranges_assemble_the_gram(q, oracle, prec, N, n, reps, world):
    from paper_2405_02630_gb300 import shard
    X = torch.from_numpy(inputs.uniform_features(N, n, 400 + N)).cuda()
    Kd, Ld = q.gram(X, reps, prec, logK=True)
    td = q.qsvm_gram_tile_dim(reps, prec)
    S = shard.padded_side(N, reps, prec)
    mps = q.qsvm_build_mps(X, reps, prec)
    outK = torch.zeros((S, S), dtype=torch.float64, device="cuda")
    outL = torch.zeros_like(outK)
    for r in range(world):
        b, e = q.qsvm_gram_partition(N, reps, prec, world, r)
        Kl = torch.full((S, S), float("nan"), dtype=torch.float64, device="cuda")
        Ll = torch.full_like(Kl, float("nan"))
        q.qsvm_kernel_gram_tiles(mps, N, n, reps, prec, b, e, Kl, logK=Ll)
        ti, tj = shard.rank_tiles(N, reps, prec, world, r)
        shard.unpack_tiles(outK, shard.pack_tiles(Kl, ti, tj, td), ti, tj, td)
        shard.unpack_tiles(outL, shard.pack_tiles(Ll, ti, tj, td), ti, tj, td)
    torch.cuda.synchronize()
    assert q.qsvm_device_status() == 0
    K = shard._mirror_upper(outK, N)
    L = shard._mirror_upper(outL, N)
    assert not torch.isnan(K).any()
    assert torch.equal(K, Kd) and torch.equal(L, Ld)
    Ko, LKo = oracle.mps_gram(X.cpu().numpy(), reps)
    _vs_oracle(K, L, Ko, LKo, prec, f"assembled shards N={N} world={world}")


def test_gram_sharded_one_rank_nccl(q, oracle):
    import torch.distributed as dist

    from paper_2405_02630_gb300 import shard
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    dist.init_process_group("nccl", init_method=f"tcp://127.0.0.1:{port}", rank=0, world_size=1,
                            device_id=torch.device("cuda", 0))
    try:
        Xh = inputs.mnist_like_features(333, 40, 12)
        X = torch.from_numpy(Xh).cuda()
        Kd, Ld = q.gram(X, 2, "fp32_split", logK=True)
        K, L = shard.gram_sharded(X, 2, "fp32_split", dst=0)
        Ka, La = shard.gram_sharded(X, 2, "fp32_split", dst=None, logK=False, stream=torch.cuda.Stream())
        torch.cuda.synchronize()
        assert torch.equal(K, Kd) and torch.equal(L, Ld)
        assert torch.equal(Ka, Kd) and La is None
        Ko, LKo = oracle.mps_gram(Xh, 2)
        _vs_oracle(K, L, Ko, LKo, "fp32_split", "gram_sharded")
    finally:
        dist.destroy_process_group()
