"""Row sharding of one preconditioner build over several ranks (one GPU each).

Sec. IV-A of the paper distributes the rows of the matrix evenly over the
processes; every process holds the whole matrix (a walk can reach any row)
and builds its own sampling tables (Sec. V-B), computes its rows of the
inverse, and the pieces are concatenated into one CSR at the end.  Here each
rank runs mcmi_build_ex on its contiguous row range [row_begin, row_end) with
the same seed -- the walks are keyed by (seed, row, chain, step), so every
row comes out exactly as in a one-rank build -- and the CSR pieces are
gathered with torch.distributed (NCCL for CUDA tensors, gloo for CPU tensors)
and concatenated in rank order.  The only exchange is that final gather.
"""
from __future__ import annotations

import numpy as np


def partition_rows(n, world, weights=None):
    """Contiguous row ranges [(begin, end)] for `world` ranks.  Without
    weights the rows are split evenly (the paper's distribution); with
    per-row weights (for example off-diagonal counts) each range holds about
    1/world of the total weight.  Ranges may be empty when n < world."""
    if world < 1 or n < 0:
        raise ValueError("world >= 1 and n >= 0 required")
    if weights is None:
        cuts = [(n * r) // world for r in range(world + 1)]
    else:
        w = np.asarray(weights, dtype=np.float64)
        if w.shape != (n,) or np.any(w < 0):
            raise ValueError("one non-negative weight per row required")
        cum = np.concatenate([[0.0], np.cumsum(w)])
        tot = cum[-1]
        if tot <= 0:
            return partition_rows(n, world)
        cuts = [0] + [int(np.searchsorted(cum, tot * r / world, side="left")) for r in range(1, world)] + [n]
        cuts = [min(max(c, 0), n) for c in cuts]
        for r in range(1, world + 1):
            cuts[r] = max(cuts[r], cuts[r - 1])
    return [(cuts[r], cuts[r + 1]) for r in range(world)]


def gather_csr(rp, col, val, group=None):
    """Concatenate the CSR pieces of all ranks in rank order.

    rp: int64[rows + 1] row pointers of this rank's rows (rp[0] == 0), col:
    int32[nnz], val: float32 or float64[nnz], all torch tensors on the
    device the process group communicates on.  Returns the whole matrix's
    (row_ptr, col, val) on every rank.  Collectives: one all-gather of the
    per-rank (rows, nnz) sizes, then one padded all-gather each of the row
    counts, columns and values."""
    import torch
    import torch.distributed as dist
    if not dist.is_initialized():   # one process: the piece is the whole matrix
        return rp, col, val
    world = dist.get_world_size(group)
    dev = rp.device
    rows = rp.numel() - 1
    nnz = col.numel()
    if int(rp[0]) != 0 or int(rp[-1]) != nnz or val.numel() != nnz:
        raise ValueError("inconsistent CSR piece")
    sizes = torch.tensor([rows, nnz], dtype=torch.int64, device=dev)
    all_sizes = [torch.empty_like(sizes) for _ in range(world)]
    dist.all_gather(all_sizes, sizes, group=group)
    all_sizes = [tuple(int(x) for x in s.tolist()) for s in all_sizes]
    max_rows = max(max(s[0] for s in all_sizes), 1)
    max_nnz = max(max(s[1] for s in all_sizes), 1)

    def padded_gather(x, length):
        buf = torch.zeros(length, dtype=x.dtype, device=dev)
        buf[:x.numel()] = x
        out = [torch.empty_like(buf) for _ in range(world)]
        dist.all_gather(out, buf, group=group)
        return out

    counts = padded_gather(rp[1:] - rp[:-1], max_rows)
    cols = padded_gather(col, max_nnz)
    vals = padded_gather(val, max_nnz)
    cnt = torch.cat([counts[r][:all_sizes[r][0]] for r in range(world)])
    row_ptr = torch.zeros(cnt.numel() + 1, dtype=torch.int64, device=dev)
    torch.cumsum(cnt, 0, out=row_ptr[1:])
    col_all = torch.cat([cols[r][:all_sizes[r][1]] for r in range(world)])
    val_all = torch.cat([vals[r][:all_sizes[r][1]] for r in range(world)])
    return row_ptr, col_all, val_all


def build_sharded(B, p, group=None, stream=None, weights=None):
    """One preconditioner build of the whole matrix B, its rows split over
    the ranks of `group`: this rank builds its row range with mcmi_build_ex
    (same parameters and seed on every rank), then the pieces are gathered.
    Returns (row_ptr, col, val, stats of this rank's build)."""
    import torch.distributed as dist
    from . import mcmi_build_ex
    world, rank = (dist.get_world_size(group), dist.get_rank(group)) if dist.is_initialized() else (1, 0)
    b, e = partition_rows(B.n, world, weights)[rank]
    q = type(p).from_buffer_copy(p)
    if e > b:
        q.row_begin, q.row_end = b, e
        M = mcmi_build_ex(B, q, stream)
        rp, col, val = M.to_torch(stream)
        rp, col, val = rp.clone(), col.clone(), val.clone()
        stats = M.stats
        M.close()
    else:
        import torch
        rp = torch.zeros(1, dtype=torch.int64, device="cuda")
        col = torch.zeros(0, dtype=torch.int32, device="cuda")
        val = torch.zeros(0, dtype=torch.float32, device="cuda")
        stats = None
    return (*gather_csr(rp, col, val, group), stats)
