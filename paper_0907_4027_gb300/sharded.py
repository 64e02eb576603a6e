"""Multi-GPU forms of the method.

Replicas: holograms are independent, so N GPUs run N holograms (or N shares of a batch) with
no data exchange; only the timing is combined (max over ranks).

Row bands (the sharded form of one hologram): Eq. 1 sums over pixels, so each rank holds a
contiguous band of rows, computes partial sums of V_m over its band, and the partial sums
are added over the ranks once per iteration (an all-reduce of 2M int64 fixed-point values:
exact, so every rank derives the same weights and coefficients, Sec. 3).  The
back-projection (Sec. 4) is local to each band.
"""
from __future__ import annotations


def band_rows(H: int, world: int, rank: int) -> tuple[int, int]:
    """(y0, rows) of rank's contiguous band when H rows are split over world ranks as evenly
    as possible (the first H % world bands get one row more)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} of {world}")
    base, extra = divmod(H, world)
    y0 = rank * base + min(rank, extra)
    return y0, base + (1 if rank < extra else 0)


def share(n: int, world: int, rank: int) -> range:
    """Indices of rank's share of n independent units (contiguous, as even as possible)."""
    y0, cnt = band_rows(n, world, rank)
    return range(y0, y0 + cnt)


def max_over_ranks(x: float, group=None) -> float:
    """Maximum of a per-rank value (e.g. a timed region's length) over the process group."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size(group) == 1:
        return float(x)
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def allreduce_exchange(group=None):
    """Exchange for run_sharded: sums a tensor in place over the process group."""
    import torch.distributed as dist

    def exchange(t):
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return exchange


def run_sharded(band, iters: int, exchange):
    """GSW with iters iterations on one row band.  band: an object with sharded_begin(),
    sharded_step(k), sharded_sums(k) -> tensor of partial sums (modified in place),
    sharded_end(iters) -> (e, u) -- a Hologram after set_band(), or any engine with that
    interface.  exchange(tensor) replaces the tensor by its sum over all bands.  Every band
    must call this with the same iters.  Returns (e, u) of the whole hologram."""
    band.sharded_begin()
    exchange(band.sharded_sums(0))
    for k in range(1, iters + 1):
        band.sharded_step(k)
        exchange(band.sharded_sums(k))
    return band.sharded_end(iters)
