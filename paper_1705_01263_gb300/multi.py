"""Several devices on one image (Sec. 3.2.2 of the paper: iteration sets are
independent, so devices render disjoint ranges of iterations into their own
films and the films are summed once at the end).

One process per GPU. `rank_iterations` splits a range of iterations
(passes over the image) into contiguous per-rank ranges; `reduce_film` sums
the FP64 film buffers (sum, sum of squares, sample count) of all ranks with
one all-reduce, the only exchange of the method; `render_distributed` puts
the two around rt_render. The reduction works on any torch.distributed
backend (NCCL on GPU buffers, gloo on CPU buffers).
"""
from __future__ import annotations


def rank_iterations(rank: int, world: int, first: int, spp: int):
    """(first_r, spp_r): the contiguous part of iterations [first, first +
    spp) that `rank` of `world` renders; the parts tile the range in rank
    order and differ in length by at most one."""
    if world < 1 or not 0 <= rank < world or spp < 0 or first < 0:
        raise ValueError("rank_iterations: invalid arguments")
    base, extra = divmod(spp, world)
    start = first + rank * base + min(rank, extra)
    return start, base + (1 if rank < extra else 0)


def reduce_film(sum_, sum2, count, group=None):
    """Sum the film buffers of all ranks in place (FP64 sums, integer
    counts). Tensors may live on the GPU (NCCL) or the CPU (gloo)."""
    import torch
    import torch.distributed as dist
    if not dist.is_initialized():
        return sum_, sum2, count
    for t in (sum_, sum2):
        if t.dtype != torch.float64:
            raise TypeError("reduce_film: the sums must be FP64")
    dist.all_reduce(sum_, op=dist.ReduceOp.SUM, group=group)
    dist.all_reduce(sum2, op=dist.ReduceOp.SUM, group=group)
    # counts: int64 for the reduction (uint32 has no all-reduce), then back
    c64 = count.to(torch.int64)
    dist.all_reduce(c64, op=dist.ReduceOp.SUM, group=group)
    count.copy_(c64.to(count.dtype))
    return sum_, sum2, count


def render_distributed(scene, cam, spp: int, max_depth: int, film, opts=None, first: int = 0, group=None):
    """Render iterations [first, first + spp) of one image across the ranks
    of `group` (each rank its own GPU and film) and sum the films into every
    rank's film."""
    import torch.distributed as dist
    from . import rt
    rank = dist.get_rank(group) if dist.is_initialized() else 0
    world = dist.get_world_size(group) if dist.is_initialized() else 1
    start, n = rank_iterations(rank, world, first, spp)
    film.seek(start)
    if n:
        rt.rt_render(scene, cam, n, max_depth, film, opts)
    s, s2, c = film.buffers()
    import torch
    torch.cuda.synchronize()
    reduce_film(s, s2, c, group)
    return film
