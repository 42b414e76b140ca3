"""Pair sharding over the ranks of a multi-GPU job: the paper's Sec. 3.2
MPI layer (divide the alignments over the ranks, align each share with the
GPU kernels, gather the results), with one process per GPU and
``torch.distributed`` for the gather.

Every rank holds the whole input (the pool and the per-pair metadata); the
partition is the library's longest-processing-time split by cells
(``nw_shard_pairs``), so every rank computes the same assignment and no
scatter is needed.  Each rank aligns its pairs with ``nw_align_batch``;
then three all-gathers give every rank every score and CIGAR: the scores
and CIGAR lengths (padded to the largest share), then the CIGAR bytes
(padded to the largest blob).  With the NCCL backend the collectives run on
CUDA tensors of the rank's device, with gloo on host tensors; no collective
reads another GPU's memory inside a kernel.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import DEFAULT_SCORING, NW_CIGAR, NWError, _u32, load, nw_align_batch


def shard_pairs(a_len, b_len, nranks: int):
    """(rank of each pair, cells per rank) by the library's LPT split."""
    al, alp = _u32(a_len)
    bl, blp = _u32(b_len)
    n = int(al.size)
    rank_of = np.zeros(max(n, 1), np.uint32)
    loads = np.zeros(max(nranks, 1), np.uint64)
    rc = load().nw_shard_pairs(alp, blp, n, nranks, rank_of.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32)),
                               loads.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
    if rc != 0:
        raise NWError(rc, "nw_shard_pairs: bad argument")
    return rank_of[:n], loads[:nranks]


def _collective_device():
    import torch
    import torch.distributed as dist
    if dist.get_backend() == "nccl":
        return torch.device("cuda", torch.cuda.current_device())
    return torch.device("cpu")


def gather_results(rank_of, rank: int, world: int, my_scores, my_cigars):
    """All-gather the per-rank results into pair order.  ``my_scores`` /
    ``my_cigars`` hold this rank's pairs in ascending pair index; returns
    (scores of every pair, CIGARs of every pair or None)."""
    import torch
    import torch.distributed as dist
    dev = _collective_device()
    npairs = int(rank_of.size)
    counts = np.bincount(rank_of, minlength=world).astype(np.int64)
    width = int(counts.max()) if npairs else 0
    want = my_cigars is not None
    # scores and CIGAR lengths of each rank's share, padded to the largest
    meta = torch.zeros((2, max(width, 1)), dtype=torch.int64, device=dev)
    meta[0, : len(my_scores)] = torch.as_tensor(np.asarray(my_scores, np.int64), device=dev)
    blob = b""
    if want:
        lens = [len(c) for c in my_cigars]
        meta[1, : len(lens)] = torch.as_tensor(np.asarray(lens, np.int64), device=dev)
        blob = "".join(my_cigars).encode()
    metas = [torch.empty_like(meta) for _ in range(world)]
    dist.all_gather(metas, meta)
    metas = [m.cpu().numpy() for m in metas]
    scores = np.zeros(npairs, np.int32)
    idx_of = [np.nonzero(rank_of == r)[0] for r in range(world)]
    for r in range(world):
        scores[idx_of[r]] = metas[r][0, : idx_of[r].size]
    if not want:
        return scores, None
    sizes = [int(metas[r][1, : idx_of[r].size].sum()) for r in range(world)]
    big = max(max(sizes), 1)
    mine = torch.zeros(big, dtype=torch.uint8, device=dev)
    if blob:
        mine[: len(blob)] = torch.frombuffer(bytearray(blob), dtype=torch.uint8).to(dev)
    blobs = [torch.empty_like(mine) for _ in range(world)]
    dist.all_gather(blobs, mine)
    cigars = [None] * npairs
    for r in range(world):
        data = blobs[r].cpu().numpy().tobytes()
        pos = 0
        for k, n in zip(idx_of[r].tolist(), metas[r][1, : idx_of[r].size].tolist()):
            cigars[k] = data[pos: pos + n].decode()
            pos += n
    return scores, cigars


def align_batch_sharded(ctx, pool2b, a_off, a_len, b_off, b_len, scoring=DEFAULT_SCORING, flags: int = 0,
                        aligner=None):
    """nw_align_batch over the ranks of the default process group: this rank
    aligns its LPT share, every rank receives every result.  ``pool2b`` is a
    host array (the share runs with NW_HOST_IO).  Returns (scores, CIGARs or
    None) in pair order, and this rank's pair indices.  ``aligner(idx)``
    replaces the library call for the share (tests of the host logic)."""
    import torch.distributed as dist
    rank, world = (dist.get_rank(), dist.get_world_size()) if dist.is_initialized() else (0, 1)
    a_off, a_len = np.asarray(a_off, np.uint64), np.asarray(a_len, np.uint32)
    b_off, b_len = np.asarray(b_off, np.uint64), np.asarray(b_len, np.uint32)
    rank_of, _ = shard_pairs(a_len, b_len, world)
    mine = np.nonzero(rank_of == rank)[0]
    if aligner is not None:
        my_scores, my_cigars = aligner(mine)
    elif mine.size:
        my_scores, my_cigars = nw_align_batch(ctx, pool2b, a_off[mine], a_len[mine], b_off[mine], b_len[mine],
                                              scoring, flags)
    else:
        my_scores, my_cigars = np.zeros(0, np.int32), ([] if flags & NW_CIGAR else None)
    if world == 1:
        return np.asarray(my_scores, np.int32), my_cigars, mine
    scores, cigars = gather_results(rank_of, rank, world, my_scores, my_cigars if flags & NW_CIGAR else None)
    return scores, cigars, mine
