"""Replica data parallelism for batches of independent states.

States are independent (one state per thread, Sec. 2.1), so a batch shards
into contiguous chunks with no exchange on the data path; a shard is simply
(pointer offset, count) on the same C ABI.  These helpers split a batch over
ranks, take the maximum of per-rank times and, for callers that want every
rank to hold all outputs, all-gather state-major outputs; the adjoint's
parameter gradient, a sum over states, is the one quantity that needs an
exchange (an all-reduce of Nr x 3 values).
"""
from __future__ import annotations


def shard(n: int, world: int, rank: int):
    """Contiguous [lo, hi) of n states for `rank` of `world` (sizes differ by <= 1)."""
    if world < 1 or not (0 <= rank < world) or n < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def max_over_ranks(value: float, dist=None) -> float:
    """Maximum of a per-rank scalar (e.g. ms per step) across the process group."""
    import torch
    if dist is None or not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    backend = dist.get_backend()
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_states(local, n_total: int, dist):
    """All-gather an output [rows, n_local] whose columns are this rank's
    contiguous shard (see shard) into [rows, n_total] on every rank."""
    import torch
    world, rank = dist.get_world_size(), dist.get_rank()
    counts = [shard(n_total, world, r)[1] - shard(n_total, world, r)[0] for r in range(world)]
    width = max(counts)
    rows = local.shape[0]
    buf = torch.zeros((rows, width), dtype=local.dtype, device=local.device)
    buf[:, : local.shape[1]] = local
    parts = [torch.empty_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf.contiguous())
    return torch.cat([p[:, :c] for p, c in zip(parts, counts)], dim=1)


def allreduce_sum(t, dist=None):
    """Sum a tensor over the process group in place (e.g. the VJP's per-shard
    parameter gradient g_theta [Nr, 3]); returns it."""
    if dist is None or not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return t
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t
