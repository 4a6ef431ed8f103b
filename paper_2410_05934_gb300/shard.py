"""Row sharding across devices (one process per GPU).

Every (polynomial, modulus) row of a batch is an independent transform
(Sec. II-D: each RNS limb of each polynomial is transformed on its own), so
a batch splits into contiguous row ranges with no exchange step.  Each rank
calls ntt_forward_rows / ntt_inverse_rows on its own range; no collective
touches the data path.  The only collectives are the timing barrier and the
max-over-ranks reduction of the measured time.
"""


def shard_rows(total_rows, rank, world):
    """Contiguous, balanced range [begin, begin + count) of rank `rank`."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank/world")
    base, extra = divmod(total_rows, world)
    begin = rank * base + min(rank, extra)
    return begin, base + (1 if rank < extra else 0)


def max_over_ranks(value, group=None):
    """max of a float over all ranks (identity without torch.distributed)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    backend = dist.get_backend(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    t = torch.tensor([float(value)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def barrier(group=None):
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier(group=group)
