"""One process per GPU, each fitting its own shard of independent surfaces.

The surfaces (or curves) of a fitting job are independent problems: their
forward, loss and gradients never mix (Sec. 3: every surface has its own
control net, knots and samples).  N GPUs therefore split a job by items and
run with no collective on the data path; per-GPU work stays fixed as N grows
(weak scaling).  The only cross-rank traffic is host-side bookkeeping: a
barrier around a timed region, the maximum of the ranks' elapsed times and the
sum of the units they processed.

Ranks are read from the usual launcher variables (RANK, WORLD_SIZE,
LOCAL_RANK, MASTER_ADDR/MASTER_PORT); without them the process is rank 0 of 1.
"""
from __future__ import annotations

import os
from dataclasses import dataclass

import torch
import torch.distributed as dist


@dataclass(frozen=True)
class Ranks:
    rank: int
    world: int
    local: int


def env() -> Ranks:
    return Ranks(int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
                 int(os.environ.get("LOCAL_RANK", "0")))


def init(backend: str) -> Ranks:
    """Join the process group when there is more than one rank."""
    r = env()
    if r.world > 1 and not dist.is_initialized():
        dist.init_process_group(backend)
    return r


def finalize():
    if dist.is_available() and dist.is_initialized():
        dist.destroy_process_group()


def shard_range(count: int, rank: int, world: int) -> tuple[int, int]:
    """Items [lo, hi) of rank `rank` when `count` items are split into `world`
    contiguous shards whose sizes differ by at most one."""
    if world < 1 or not 0 <= rank < world or count < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(count, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def shard_seed(seed: int, rank: int) -> int:
    """Seed of rank `rank`'s synthetic shard (distinct per rank, fixed per run)."""
    return seed + 1_000_003 * rank


def barrier():
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def _reduce(x: float, op, device) -> float:
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=op)
    return float(t.item())


def max_over_ranks(x: float, device=None) -> float:
    """Largest value of x over all ranks (the job's elapsed time)."""
    return _reduce(x, dist.ReduceOp.MAX, device)


def sum_over_ranks(x: float, device=None) -> float:
    """Sum of x over all ranks (units the whole job processed)."""
    return _reduce(x, dist.ReduceOp.SUM, device)


def job_rate(units: float, elapsed_s: float, device=None) -> float:
    """Whole-job throughput: all ranks' units over the slowest rank's time."""
    total = sum_over_ranks(units, device)
    slowest = max_over_ranks(elapsed_s, device)
    return total / slowest if slowest > 0 else 0.0
