"""Host-side logic of multi-GPU runs.  The solve shards over slices with no
exchange on the data path: every rank holds a replica of the factors (the
QR is repeated per rank, or loaded from a checkpoint) and solves its own
slices; the only collectives are the timing reduction and, when a caller
wants the whole batch on one rank, a gather of the images.  Works with any
torch.distributed backend (NCCL on GPUs, gloo on CPU)."""
from __future__ import annotations


def rank_slices(rank: int, world: int, k_per_rank: int, base_seed: int) -> tuple[int, int]:
    """(first global slice index, first phantom seed) of a rank's k slices:
    rank r owns global slices [r k, (r+1) k), seeded base_seed + r k."""
    if not (0 <= rank < world) or k_per_rank < 0:
        raise ValueError("bad rank/world/k")
    first = rank * k_per_rank
    return first, base_seed + first


def max_over_ranks(value: float, dist=None, device=None) -> float:
    """The maximum of a per-rank scalar (the step time of the slowest rank)."""
    if dist is None:
        return float(value)
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_slices(X, dist=None, dst: int = 0):
    """Concatenate the ranks' (k, n) image blocks in rank order on rank dst
    (None elsewhere).  Equal k on every rank."""
    if dist is None:
        return X
    import torch
    world = dist.get_world_size()
    if dist.get_rank() == dst:
        parts = [torch.empty_like(X) for _ in range(world)]
        dist.gather(X, gather_list=parts, dst=dst)
        return torch.cat(parts, dim=0)
    dist.gather(X, dst=dst)
    return None
