"""Y-slab decomposition of one grid over the ranks of a process group: the
exchange step of a single large solve spread over several GPUs.

The substep's stencil reaches two cells each way (MinMod reconstruction of
the face states, Sec. 2.1 step 1; the velocity gradients reach one), and the
source and frequency steps are cell-local.  So rank r owns rows [y0, y1) and
keeps HALO = 2 rows of each neighbour around them; before every substep the
ranks swap their edge rows, every rank advances its extended slab with the
same (global) time step, and its own rows then come out exactly as in a
single-domain run: they depend only on rows the rank holds correctly.  The
halo rows come out wrong (their own stencil reaches beyond the slab) and are
overwritten by the next swap.

Domain-wide quantities reduce across the slabs: the time step (global_dt)
and the dynamic reduced speed of light (global_ctilde).  Active-bin pruning
decides on the domain's energy per bin, which no slab holds, so slab runs
keep it off.

The module is solver-agnostic: state arrays are [nb][rows][nx] numpy arrays
or torch tensors (CPU with gloo, CUDA with NCCL); the caller advances its
slab with whatever it uses.  A lym1 context swaps only its halo rows, in
its own element type and on the device, with exchange_ctx (lym1_get_rows /
lym1_set_rows), so no full state leaves the GPU between substeps.
"""
import numpy as np
import torch
import torch.distributed as dist

HALO = 2


def slab_rows(ny: int, world: int, rank: int):
    """Rows [y0, y1) owned by rank: a balanced split, sizes differing by at most one."""
    base, extra = divmod(ny, world)
    y0 = rank * base + min(rank, extra)
    return y0, y0 + base + (1 if rank < extra else 0)


def extended_rows(ny: int, world: int, rank: int):
    """Rows [e0, e1) the rank holds: its own plus up to HALO of each neighbour."""
    y0, y1 = slab_rows(ny, world, rank)
    return max(0, y0 - HALO), min(ny, y1 + HALO)


def check_split(ny: int, world: int):
    """Every slab must hold at least HALO rows, so that a neighbour's halo
    comes from a single rank."""
    for r in range(world):
        y0, y1 = slab_rows(ny, world, r)
        if y1 - y0 < HALO:
            raise ValueError(f"{ny} rows over {world} ranks leaves rank {r} fewer than {HALO} rows")


def _as_tensor(a):
    return a if isinstance(a, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(a))


def exchange(arrays, ny: int, world: int, rank: int, group=None):
    """Swap the halo rows of the extended-slab arrays ([nb][e1 - e0][nx]) in
    place: this rank's lowest and highest HALO own rows go to the ranks below
    and above, whose edge rows fill this rank's halo."""
    if world == 1:
        return
    y0, y1 = slab_rows(ny, world, rank)
    e0, e1 = extended_rows(ny, world, rank)
    lo, hi = y0 - e0, y1 - e0  # own rows, relative to the extended slab
    for a in arrays:
        t = _as_tensor(a)
        reqs, recvs = [], []
        if rank > 0:
            reqs.append(dist.isend(t[:, lo:lo + HALO].contiguous(), rank - 1, group=group))
            buf = torch.empty_like(t[:, 0:lo].contiguous())
            reqs.append(dist.irecv(buf, rank - 1, group=group))
            recvs.append((slice(0, lo), buf))
        if rank < world - 1:
            reqs.append(dist.isend(t[:, hi - HALO:hi].contiguous(), rank + 1, group=group))
            buf = torch.empty_like(t[:, hi:].contiguous())
            reqs.append(dist.irecv(buf, rank + 1, group=group))
            recvs.append((slice(hi, t.shape[1]), buf))
        for r in reqs:
            r.wait()
        for rows, buf in recvs:
            if isinstance(a, torch.Tensor):
                a[:, rows].copy_(buf)
            else:
                a[:, rows] = buf.numpy()


def exchange_ctx(ctx, ny: int, world: int, rank: int, group=None, device=None):
    """Swap the halo rows of a slab solver in place through its row calls:
    ``ctx`` holds this rank's extended rows [e0, e1) and offers
    ``get_rows(y0, n, out)`` / ``set_rows(y0, J, Hx, Hy)`` over [nb][n][nx]
    buffers of its state's element type (a lym1 context: lym1_get_rows /
    lym1_set_rows, ``ctx.state_itemsize()`` bytes per element).  Only the
    2 x HALO edge rows travel: this rank's lowest and highest HALO own rows go
    to the ranks below and above, whose edge rows land in this rank's halo.
    ``device``: where the row buffers live (a CUDA device for NCCL, the CPU
    for gloo); the row calls copy between it and the solver's state."""
    if world == 1:
        return
    y0, y1 = slab_rows(ny, world, rank)
    e0, e1 = extended_rows(ny, world, rank)
    lo, hi = y0 - e0, y1 - e0  # own rows, relative to the extended slab
    dtype = torch.float32 if ctx.state_itemsize() == 4 else torch.float64
    dev = torch.device("cpu") if device is None else torch.device(device)

    def buf(n):
        return tuple(torch.empty((ctx.nb, n, ctx.nx), dtype=dtype, device=dev) for _ in range(3))

    reqs, recvs = [], []
    if rank > 0:
        send = ctx.get_rows(lo, HALO, buf(HALO))
        reqs += [dist.isend(t, rank - 1, group=group) for t in send]
        r = buf(lo)
        reqs += [dist.irecv(t, rank - 1, group=group) for t in r]
        recvs.append((0, r))
    if rank < world - 1:
        send = ctx.get_rows(hi - HALO, HALO, buf(HALO))
        reqs += [dist.isend(t, rank + 1, group=group) for t in send]
        r = buf(e1 - e0 - hi)
        reqs += [dist.irecv(t, rank + 1, group=group) for t in r]
        recvs.append((hi, r))
    for q in reqs:
        q.wait()
    if dev.type == "cuda":
        torch.cuda.current_stream(dev).synchronize()  # the received rows, before the solver's stream reads them
    for row0, (J, Hx, Hy) in recvs:
        ctx.set_rows(row0, J, Hx, Hy)


def global_ctilde(local_ctilde: float, group=None) -> float:
    """The single-domain dynamic reduced speed of light (Sec. 2.1, the
    dynamic-RSL rule): each slab applies the rule to its own cells from the
    same previous value.  The rule is a maximum over cells followed by the
    floor, the cap and the rate limits, all non-decreasing, so the domain's
    value is the largest of the slabs' values.  Every slab then takes it
    (set_ctilde), which keeps the previous values equal for the next update."""
    t = torch.tensor([float(local_ctilde)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def global_dt(local_dt: float, group=None) -> float:
    """The single-domain CFL step: the smallest of the slabs' own steps (each
    slab sees a subset of the velocities, and every cell is in some slab)."""
    t = torch.tensor([float(local_dt)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MIN, group=group)
    return float(t.item())
