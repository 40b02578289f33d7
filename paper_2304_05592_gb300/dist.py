"""Shot-parallel gradients over ranks (one process per GPU).

The misfit and its gradient are sums over shots, and every shot is an
independent wave solve (arxiv 2304.05592, section "Putting it all together":
gradients over randomly selected shots).  So a survey is split into one
contiguous range of shots per rank, each rank runs the batched solver on its
range, and one all-reduce of the gradient (plus the scalar misfit) is the
only exchange.  The solver is passed in as a callable, so the same code runs
the CUDA library on GPUs (NCCL) and any other implementation of a gradient on
CPU ranks (gloo).
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def shard(nshot: int, rank: int, world: int) -> range:
    """The shots of `rank`: contiguous ranges whose sizes differ by at most one."""
    if world < 1 or not 0 <= rank < world or nshot < 0:
        raise ValueError(f"bad shard request: nshot={nshot} rank={rank} world={world}")
    base, extra = divmod(nshot, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def world_info():
    if dist.is_available() and dist.is_initialized():
        return dist.get_rank(), dist.get_world_size()
    return 0, 1


def sharded_gradient(grad_fn, nshot: int, out: torch.Tensor | None = None):
    """Misfit and gradient summed over all nshot shots of the survey.

    grad_fn(shots) returns (misfit, gradient tensor) for a range of shot
    indices (an empty range must return zeros).  The gradient is summed over
    ranks in place with one all-reduce; the misfit rides along in the same
    call as one extra element, so the exchange is a single collective."""
    rank, world = world_info()
    phi, g = grad_fn(shard(nshot, rank, world))
    if world == 1:
        return float(phi), g
    buf = torch.cat([g.reshape(-1).to(torch.float64), torch.tensor([float(phi)], dtype=torch.float64,
                                                                    device=g.device)])
    dist.all_reduce(buf)
    g_sum = buf[:-1].to(g.dtype).reshape(g.shape)
    if out is not None:
        out.copy_(g_sum)
        g_sum = out
    return float(buf[-1].item()), g_sum
