"""Multi-process helpers: one process per GPU.

The chains of a batch are independent, and so are replicas of a single-chain workload, so the
benchmark's ranks exchange no data on the hot path: the only collectives are a barrier around
the timed region and a max-reduction of the elapsed time.

A single chain split across ranks is the sub-domain decomposition of the library's
rk4_domain_* calls with one part per rank: each rank holds its part with ghost zones (the
library's layout, from rk4_domain_part) and integrates it as a fixed-end chain; every
floor(ghost / reach) steps the ranks swap ghost zones with their neighbours by point-to-point
messages (exchange_ghosts, integrate_decomposed).  reach = stages x coupling range sites per
step (4 for classical RK4 with nearest neighbours).
"""
from __future__ import annotations

import os


def env_rank() -> tuple[int, int, int]:
    """(rank, world_size, local_rank) from the torchrun environment (defaults: single process)."""
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def init(backend: str = "nccl"):
    """Initialise torch.distributed when WORLD_SIZE > 1; returns (rank, world, local_rank)."""
    import torch.distributed as dist
    rank, world, local = env_rank()
    if world > 1 and not dist.is_initialized():
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        os.environ.setdefault("MASTER_PORT", "29511")
        dist.init_process_group(backend=backend, rank=rank, world_size=world)
    return rank, world, local


def barrier():
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.barrier()


def max_over_ranks(x: float) -> float:
    """The largest value of x over all ranks (the job's elapsed time)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    backend = dist.get_backend()
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    backend = dist.get_backend()
    dev = torch.device("cuda", torch.cuda.current_device()) if backend == "nccl" else torch.device("cpu")
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def shard_chains(lengths, world: int, rank: int):
    """Indices of the chains rank `rank` integrates: longest-processing-time-first bin packing
    by chain length (work is proportional to sites), deterministic on every rank."""
    order = sorted(range(len(lengths)), key=lambda i: (-int(lengths[i]), i))
    load = [0] * world
    owner = [0] * len(lengths)
    for i in order:
        r = min(range(world), key=lambda j: (load[j], j))
        owner[i] = r
        load[r] += int(lengths[i])
    return [i for i in range(len(lengths)) if owner[i] == rank]


def neighbours(rank: int, world: int, periodic: bool):
    """(left, right) neighbour ranks of `rank`'s part; None at a fixed end."""
    left = (rank - 1) % world if (periodic or rank > 0) else None
    right = (rank + 1) % world if (periodic or rank < world - 1) else None
    return left, right


def exchange_ghosts(ext, part: dict, ghost: int, left, right):
    """Refresh the ghost zones of this rank's block `ext` ([ghost_left + sites + ghost_right, D],
    a torch tensor on the backend's device; `part` as rk4_domain_part returns it) from the
    neighbour ranks: the left ghosts become the left neighbour's last `ghost` sites, the right
    ghosts the right neighbour's first `ghost` sites.  A neighbour equal to this rank (a single
    periodic part) is copied locally."""
    import torch.distributed as dist
    gl, n = part["ghost_left"], part["sites"]
    first = ext[gl:gl + ghost]
    last = ext[gl + n - ghost:gl + n]
    rank = dist.get_rank() if (dist.is_available() and dist.is_initialized()) else 0
    reqs, recvs = [], []
    # tag 0: sites travelling right (into a left ghost zone); tag 1: travelling left
    if right is not None and right != rank:
        reqs.append(dist.isend(last.contiguous(), right, tag=0))
    if left is not None and left != rank:
        reqs.append(dist.isend(first.contiguous(), left, tag=1))
    if left is not None:
        if left == rank:
            ext[:gl].copy_(last)
        else:
            buf = ext.new_empty((gl,) + tuple(ext.shape[1:]))
            reqs.append(dist.irecv(buf, left, tag=0))
            recvs.append((buf, slice(0, gl)))
    if right is not None:
        if right == rank:
            ext[gl + n:].copy_(first)
        else:
            buf = ext.new_empty((part["ghost_right"],) + tuple(ext.shape[1:]))
            reqs.append(dist.irecv(buf, right, tag=1))
            recvs.append((buf, slice(gl + n, gl + n + part["ghost_right"])))
    for r in reqs:
        r.wait()
    for buf, sl in recvs:
        ext[sl].copy_(buf)


def exchange_ghosts_host(ext, part: dict, ghost: int, left, right):
    """exchange_ghosts for a block held in device memory when the process group's backend moves
    host tensors (gloo): only the block's edges travel through host memory -- its two ghost
    zones and the `ghost` sites next to each -- and the received ghost zones are copied back."""
    import torch
    gl, n, gr = part["ghost_left"], part["sites"], part["ghost_right"]
    if n >= 2 * ghost:
        small = torch.cat([ext[:gl + ghost].cpu(), ext[gl + n - ghost:].cpu()])
        small_part = {"ghost_left": gl, "sites": 2 * ghost, "ghost_right": gr}
    else:
        small = ext.cpu()
        small_part = part
    exchange_ghosts(small, small_part, ghost, left, right)
    if gl:
        ext[:gl].copy_(small[:gl])
    if gr:
        ext[gl + n:].copy_(small[small.shape[0] - gr:])


def integrate_decomposed(ext, comp, part: dict, ghost: int, reach: int, nsteps: int, integrate, left, right,
                         exchange=exchange_ghosts):
    """Advance this rank's part nsteps steps: swap ghost zones, run `integrate(ext, comp, m)` for
    m = min(floor(ghost / reach), steps left) steps on the part as a fixed-end chain, repeat.
    On a GPU `integrate` is rk4_chain_integrate on a fixed-end handle of the block's length, and
    `exchange` is exchange_ghosts (a device-capable backend) or exchange_ghosts_host (gloo)."""
    period = ghost // reach if (left is not None or right is not None) else max(nsteps, 1)
    if period < 1:
        raise ValueError("ghost zones narrower than one step's reach")
    done = 0
    while done < nsteps:
        m = min(period, nsteps - done)
        exchange(ext, part, ghost, left, right)
        if comp is not None:
            exchange(comp, part, ghost, left, right)
        integrate(ext, comp, m)
        done += m
