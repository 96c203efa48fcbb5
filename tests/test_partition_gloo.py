"""Multi-rank Gram sharding on CPU ranks (gloo, world size 2 and 3).

Sec. 5 of the paper distributes the data pairs evenly over GPUs and gathers the
kernel pieces to one place.  Here each rank takes the tile range that
qsvm_gram_partition assigns it and contracts those pairs with the CPU oracle (standing
in for the kernel, which writes the same tiles and mirrors); the library's gather
(shard.gather_gram: pack the rank's tiles, one gather or all-gather, unpack and mirror)
assembles the Gram, which must equal the single-rank Gram bit-exactly, with every
unique pair computed by exactly one rank, also when some ranks own no tile.
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
    from paper_2405_02630_gb300 import inputs, qsvm, shard
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    X = inputs.uniform_features(N, n, 9)
    td = qsvm.qsvm_gram_tile_dim(reps, "fp32_split")
    T = -(-N // td)
    b, e = qsvm.qsvm_gram_partition(N, reps, "fp32_split", world, rank)
    pairs = [p for t in range(b, e) for p in _tile_to_pairs(t, N, T, td)]
    S = shard.padded_side(N, reps, "fp32_split")
    # the kernel's contract for a tile range: both K[i][j] and its mirror, nothing else
    K = np.full((S, S), np.nan)
    L = np.full((S, S), np.nan)
    C = np.zeros((N, N))
    if pairs:
        ia = np.array([p[0] for p in pairs])
        ib = np.array([p[1] for p in pairs])
        Kp, Lp = oracle.mps_pairs(X, X, ia, ib, reps, threads=1)
        K[ia, ib] = Kp
        K[ib, ia] = Kp
        L[ia, ib] = Lp
        L[ib, ia] = Lp
        C[ia, ib] += 1
    Ct = torch.from_numpy(C)
    dist.all_reduce(Ct)
    Kg, Lg = shard.gather_gram(torch.from_numpy(K), N, reps, "fp32_split", dst=0, logK_local=torch.from_numpy(L))
    assert (Kg is None) == (rank != 0) and (Lg is None) == (rank != 0)
    Ka, _ = shard.gather_gram(torch.from_numpy(K), N, reps, "fp32_split", dst=None)
    np.save(os.path.join(out_dir, f"Kall{rank}.npy"), Ka.numpy())
    if rank == 0:
        np.save(os.path.join(out_dir, "K.npy"), Kg.numpy())
        np.save(os.path.join(out_dir, "L.npy"), Lg.numpy())
        np.save(os.path.join(out_dir, "C.npy"), Ct.numpy())
    dist.barrier()
    dist.destroy_process_group()


def _run(tmp_path, world, N, n, reps):
    import socket

    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mp.start_processes(_worker, args=(world, port, N, n, reps, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")


@pytest.mark.parametrize("world,N", [(2, 45), (3, 45), (3, 20), (4, 61)])
def test_sharded_gram_matches_single_rank(tmp_path, oracle, world, N):
    """N = 20 at reps = 2 is two tile rows, three tiles: with three ranks one rank may own
    none, and the gather still assembles the Gram."""
    n, reps = 9, 2
    _run(tmp_path, world, N, n, reps)
    K = np.load(tmp_path / "K.npy")
    L = np.load(tmp_path / "L.npy")
    C = np.load(tmp_path / "C.npy")
    from paper_2405_02630_gb300 import inputs
    X = inputs.uniform_features(N, n, 9)
    Kref, Lref = oracle.mps_gram(X, reps)
    assert np.array_equal(np.triu(C), np.triu(np.ones((N, N))))
    assert np.array_equal(K, Kref) and np.array_equal(L, Lref)
    for r in range(world):
        assert np.array_equal(np.load(tmp_path / f"Kall{r}.npy"), Kref)


def test_pack_unpack_round_trip():
    """Packing the tiles of every rank and unpacking them into an empty buffer puts every
    value of the upper triangle back where it was, and the mirror completes the Gram."""
    from paper_2405_02630_gb300 import qsvm, shard
    N, reps, prec = 70, 2, "fp32_split"
    td = qsvm.qsvm_gram_tile_dim(reps, prec)
    S = shard.padded_side(N, reps, prec)
    rng = np.random.default_rng(0)
    A = rng.standard_normal((S, S))
    A = A + A.T
    out = torch.zeros((S, S), dtype=torch.float64)
    seen = 0
    for r in range(4):
        ti, tj = shard.rank_tiles(N, reps, prec, 4, r)
        assert np.all(ti <= tj)
        seen += len(ti)
        shard.unpack_tiles(out, shard.pack_tiles(torch.from_numpy(A), ti, tj, td), ti, tj, td)
    assert seen == qsvm.qsvm_gram_num_tiles(N, reps, prec)
    Ksym = shard._mirror_upper(out, N).numpy()
    assert np.array_equal(Ksym, A[:N, :N])
    ti, tj = qsvm.qsvm_gram_tile_list(N, reps, prec, 0, qsvm.qsvm_gram_num_tiles(N, reps, prec))
    assert [qsvm.qsvm_gram_tile_coords(N, reps, prec, b) for b in range(len(ti))] == list(zip(ti, tj))
