"""One Gram shared by several ranks, one GPU each (Sec. 5: the data pairs are spread evenly
over the GPUs and the kernel pieces are gathered to one place).

Each rank contracts the contiguous range of pair tiles that qsvm_gram_partition assigns it
(whole tiles, near-equal pair counts) into a rank-local K, packs its tiles densely as
[tiles, td, td] and the packed buffers travel in ONE collective: a gather to the owner rank,
or an all-gather when every rank needs K.  The receiver places each tile at its (ti, tj)
and mirrors the strict upper triangle, so the result is bit-identical to the single-rank
Gram.  Every rank rebuilds the MPS of all points: the build costs a small fraction of the
pair work and needs no exchange.  The tile lists are recomputed on every rank by the same
host functions, so only the packed values travel.

torch.distributed is the transport (NCCL for CUDA tensors, gloo for CPU tensors); the
contraction itself is the library's kernel.
"""
import numpy as np

from . import qsvm


def padded_side(n_points: int, reps: int, precision) -> int:
    """Side of the rank-local K buffer: n_points rounded up to whole tiles."""
    td = qsvm.qsvm_gram_tile_dim(reps, precision)
    return -(-n_points // td) * td


def rank_tiles(n_points: int, reps: int, precision, world: int, rank: int):
    """(ti, tj) int64 arrays of the tiles rank `rank` of `world` computes."""
    b, e = qsvm.qsvm_gram_partition(n_points, reps, precision, world, rank)
    return qsvm.qsvm_gram_tile_list(n_points, reps, precision, b, e)


def pack_tiles(K, ti, tj, td: int):
    """Tiles (ti[m], tj[m]) of a square (T*td, T*td) tensor as one [m, td, td] tensor."""
    import torch
    T = K.shape[0] // td
    ii = torch.as_tensor(np.asarray(ti), dtype=torch.int64, device=K.device)
    jj = torch.as_tensor(np.asarray(tj), dtype=torch.int64, device=K.device)
    return K.view(T, td, T, td)[ii, :, jj, :]


def unpack_tiles(K, packed, ti, tj, td: int):
    """Writes packed[m] at tile (ti[m], tj[m]) of a square (T*td, T*td) tensor."""
    import torch
    if len(ti) == 0:
        return K
    T = K.shape[0] // td
    ii = torch.as_tensor(np.asarray(ti), dtype=torch.int64, device=K.device)
    jj = torch.as_tensor(np.asarray(tj), dtype=torch.int64, device=K.device)
    K.view(T, td, T, td)[ii, :, jj, :] = packed
    return K


def _mirror_upper(M, n_points: int):
    """The n_points x n_points symmetric matrix whose upper triangle (with diagonal) is M's."""
    import torch
    U = torch.triu(M[:n_points, :n_points])
    return U + torch.triu(U, 1).T


def gather_gram(K_local, n_points: int, reps: int, precision, dst=0, group=None, logK_local=None):
    """Collects the tiles every rank computed into the full Gram.

    K_local (and logK_local, if given): this rank's (S, S) buffer, S = padded_side(...),
    holding at least the tiles of its range (the kernels also write the mirror, which is
    not sent).  dst: the receiving rank (a rank of the default group), or None for every
    rank.  Returns (K, logK or None) as n_points x n_points tensors on K_local's device on
    the receiving rank(s), and (None, None) elsewhere.
    """
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    me = dist.get_rank(group)
    td = qsvm.qsvm_gram_tile_dim(reps, precision)
    S = padded_side(n_points, reps, precision)
    if K_local.shape != (S, S) or (logK_local is not None and logK_local.shape != (S, S)):
        raise ValueError(f"local buffers must be ({S}, {S})")
    lists = [rank_tiles(n_points, reps, precision, world, r) for r in range(world)]
    m = max(1, max(len(t[0]) for t in lists))
    ch = 1 if logK_local is None else 2
    send = torch.zeros((m, ch, td, td), dtype=torch.float64, device=K_local.device)
    ti, tj = lists[me]
    if len(ti):
        send[:len(ti), 0] = pack_tiles(K_local, ti, tj, td)
        if ch == 2:
            send[:len(ti), 1] = pack_tiles(logK_local, ti, tj, td)
    if dst is None:
        receiving = True
    else:
        receiving = (dist.get_global_rank(group, me) if group is not None else me) == dst
    recv = [torch.empty_like(send) for _ in range(world)] if receiving else None
    if dst is None:
        dist.all_gather(recv, send, group=group)
    else:
        dist.gather(send, gather_list=recv, dst=dst, group=group)
    if not receiving:
        return None, None
    out = [torch.zeros((S, S), dtype=torch.float64, device=K_local.device) for _ in range(ch)]
    for r, (ri, rj) in enumerate(lists):
        for c in range(ch):
            unpack_tiles(out[c], recv[r][:len(ri), c], ri, rj, td)
    K = _mirror_upper(out[0], n_points)
    return K, (_mirror_upper(out[1], n_points) if ch == 2 else None)


def gram_sharded(X, reps: int, precision, dst=0, group=None, logK: bool = True, stream=None):
    """The Gram of X (CUDA float64, n_points x n_qubits, every rank the same X) computed by
    all ranks of `group` together and gathered to `dst` (None: to every rank).  Each rank
    builds the MPS of all points, contracts its partition of the pair tiles, and takes part
    in one gather.  Returns (K, logK or None) on the receiving rank(s), (None, None)
    elsewhere."""
    import torch
    import torch.distributed as dist
    N, n = X.shape
    world = dist.get_world_size(group)
    me = dist.get_rank(group)
    S = padded_side(N, reps, precision)
    b, e = qsvm.qsvm_gram_partition(N, reps, precision, world, me)
    Kl = torch.zeros((S, S), dtype=torch.float64, device=X.device)
    Ll = torch.zeros((S, S), dtype=torch.float64, device=X.device) if logK else None
    if stream is not None:
        stream.wait_stream(torch.cuda.current_stream(X.device))
    mps = qsvm.qsvm_build_mps(X, reps, precision, stream=stream)
    qsvm.qsvm_kernel_gram_tiles(mps, N, n, reps, precision, b, e, Kl, logK=Ll, stream=stream)
    if stream is not None:
        torch.cuda.current_stream(X.device).wait_stream(stream)
    return gather_gram(Kl, N, reps, precision, dst=dst, group=group, logK_local=Ll)
