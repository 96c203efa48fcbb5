"""Multi-rank Gram sharding on CPU ranks (gloo, world size 2 and 3).

Sec. 5 of the paper distributes the data pairs evenly over GPUs and gathers the
kernel pieces to one place.  Here each rank takes the tile range that
qsvm_gram_partition assigns it, contracts those pairs with the CPU oracle and the
pieces are all-gathered; the union must equal the single-rank Gram bit-exactly,
with every unique pair computed by exactly one rank.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _tile_to_pairs(b, N, T, td):
    from paper_2405_02630_gb300 import qsvm
    ti, tj = qsvm.qsvm_gram_tile_coords(N, 2, "fp32_split", b)
    pairs = []
    for i in range(ti * td, min(N, (ti + 1) * td)):
        for j in range(tj * td, min(N, (tj + 1) * td)):
            if ti != tj or i <= j:
                pairs.append((i, j))
    return pairs


def _worker(rank, world, port, N, n, reps, out_dir):
    import torch.distributed as dist

    from oracle import oracle
    from paper_2405_02630_gb300 import inputs, qsvm
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    X = inputs.uniform_features(N, n, 9)
    td = qsvm.qsvm_gram_tile_dim(reps, "fp32_split")
    T = -(-N // td)
    b, e = qsvm.qsvm_gram_partition(N, reps, "fp32_split", world, rank)
    pairs = [p for t in range(b, e) for p in _tile_to_pairs(t, N, T, td)]
    K = np.zeros((N, N))
    C = np.zeros((N, N))
    if pairs:
        ia = np.array([p[0] for p in pairs])
        ib = np.array([p[1] for p in pairs])
        Kp, _ = oracle.mps_pairs(X, X, ia, ib, reps, threads=1)
        K[ia, ib] = Kp
        K[ib, ia] = Kp
        C[ia, ib] += 1
    Kt = torch.from_numpy(K)
    Ct = torch.from_numpy(C)
    gathered = [torch.zeros_like(Kt) for _ in range(world)]
    dist.all_gather(gathered, Kt)
    dist.all_reduce(Ct)
    if rank == 0:
        # each entry comes from exactly one rank: take it from the rank that owns it
        np.save(os.path.join(out_dir, "K.npy"), sum(g.numpy() * (g.numpy() != 0) for g in gathered))
        np.save(os.path.join(out_dir, "C.npy"), Ct.numpy())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_gram_matches_single_rank(tmp_path, oracle, world):
    import socket

    import torch.multiprocessing as mp
    N, n, reps = 45, 9, 2
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mp.start_processes(_worker, args=(world, port, N, n, reps, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    K = np.load(tmp_path / "K.npy")
    C = np.load(tmp_path / "C.npy")
    from paper_2405_02630_gb300 import inputs
    X = inputs.uniform_features(N, n, 9)
    Kref, _ = oracle.mps_gram(X, reps)
    assert np.array_equal(np.triu(C), np.triu(np.ones((N, N))))
    assert np.array_equal(K, Kref)
