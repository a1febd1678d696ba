"""Host-side logic of multi-GPU runs (one process per GPU, torch.distributed).

The peel shards by cadence: each GPU owns its own channel group / cadence (the
paper's per-GPU channel sets, weak scaling across GPUs) and needs no data-path
collective.  What the ranks share is bookkeeping: a per-rank seed, a barrier
around the timed region, the slowest rank's time and the job total.

For a cadence split by channel across GPUs (Section 3.1: channel groups on
separate workers, combined centrally), every rank peels its channels with the
library's channel-shard calls and the ranks sum their partial averages once
per block of sources before the block's solve: `run_sharded_cadence` drives
that loop with any in-place sum (`sum_over_ranks`: an all-reduce over the
process group); `combine_partial_averages` scales and sums a per-rank mean.  The
ionospheric offset fit is the exchange the paper itself plans (Section 3.1:
six numbers per source from every worker, two-number solution built
centrally): `combine_offset_statistics` sums the six numbers over ranks.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def world() -> tuple[int, int]:
    """(rank, world_size); (0, 1) outside torch.distributed."""
    if dist.is_available() and dist.is_initialized():
        return dist.get_rank(), dist.get_world_size()
    return 0, 1


def rank_seed(base_seed: int, rank: int) -> int:
    """Independent cadence per rank."""
    return int(base_seed) + 1000 * int(rank)


def barrier() -> None:
    if world()[1] > 1:
        dist.barrier()


def max_over_ranks(x: float, device: str | torch.device = "cpu") -> float:
    """The slowest rank's value (the job's time)."""
    if world()[1] == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, seconds_max: float, world_size: int) -> float:
    """Whole-job throughput of weakly scaled replicas: all ranks' units over the slowest time."""
    return world_size * units_per_rank / seconds_max


def combine_partial_averages(partial: torch.Tensor, n_local: int, n_total: int) -> torch.Tensor:
    """Sum over ranks of n_local / n_total * partial (in place, returned).

    `partial` is this rank's mean over its own samples; the result is the mean
    over all samples of all ranks."""
    partial.mul_(float(n_local) / float(n_total))
    if world()[1] > 1:
        dist.all_reduce(partial, op=dist.ReduceOp.SUM)
    return partial


def combine_offset_statistics(six: torch.Tensor) -> torch.Tensor:
    """Sum over ranks of the six numbers per source [K][6] (in place, returned).

    Each rank holds a group of channels and gets (H_ll, H_lm, H_mm, g_l, g_m, L)
    from Peeler.offsets with a common nu_ref; all six are sums over channels,
    so their sum over ranks is the whole band's, ready for offsets_solve
    (Section 3.1: workers send six numbers per source, the master solves for two)."""
    if world()[1] > 1:
        dist.all_reduce(six, op=dist.ReduceOp.SUM)
    return six


def sum_over_ranks(t: torch.Tensor) -> torch.Tensor:
    """In-place sum over ranks (the exchange of a channel-sharded cadence)."""
    if world()[1] > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t


def run_sharded_cadence(begin, partials, step, exchange) -> int:
    """One channel-shard cadence: begin(); then, until step() returns 0, the
    current partial averages (partials(), a tensor) are summed in place over
    the band's shards by exchange() and step() solves and subtracts a block and
    leaves the next block's partials.  Returns the number of exchanges."""
    begin()
    n = 0
    while True:
        exchange(partials())
        n += 1
        if step() == 0:
            return n
