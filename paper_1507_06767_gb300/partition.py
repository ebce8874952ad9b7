"""Slab decomposition of one lattice over several processes (one GPU each): the plan and the host
side of its exchanges.

The fused step of Sec. 2.2 is local: a cell pulls only from its nearest neighbours, so a lattice
cut into slabs along its slowest axis (z for D3Q19, y for D2Q9) needs, per step, one plane of
populations from each neighbouring slab: the populations whose velocity crosses the cut (5 per
face for D3Q19, 3 for D2Q9).  Block maxima stay local when the cuts fall on block edges; the
top-fraction flags need the maxima of all blocks (an all-gather), and the conservation sums an
all-reduce.

The library steps a slab through its halo faces (lbm_set_halo / lbm_halo_export /
lbm_halo_import in include/lbm.h): a handle per slab whose cut faces read the neighbour's boundary
plane from a halo instead of a wall.  This module holds the plan (which ranks own which planes,
what crosses each cut) and the exchanges, written against torch.distributed so that the same code
moves CPU tensors over gloo or CUDA tensors over NCCL: `exchange_lattice_halos` for library slabs
(host-staged messages), `exchange_halos` for a slab stored with ghost planes in a tensor.
"""
from __future__ import annotations

from dataclasses import dataclass

# velocity components along the slab axis, in the library's population order (the layout of
# lbm_get_populations): D2Q9 rest, +x, +y, -x, -y, then the diagonals; D3Q19 rest, +-x, +-y, +-z,
# then the edge directions in opposite pairs
_D2Q9_CY = (0, 0, 1, 0, -1, 1, 1, -1, -1)
_D3Q19_CZ = (0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1)


def slab_velocity(q: int):
    """Component of each population's velocity along the slab axis."""
    if q == 9:
        return _D2Q9_CY
    if q == 19:
        return _D3Q19_CZ
    raise ValueError("q must be 9 or 19")


@dataclass(frozen=True)
class Slab:
    rank: int
    lo: int          # first plane owned (global index along the slab axis)
    hi: int          # one past the last plane owned
    below: int | None  # rank owning plane lo - 1 (None: a wall)
    above: int | None  # rank owning plane hi (None: a wall)


def plan(n_slow: int, world: int, align: int, periodic: bool):
    """Cut n_slow planes into `world` slabs whose cuts fall on multiples of `align` (the block edge,
    so block maxima stay local); the blocks are shared out as evenly as possible."""
    if world < 1 or align < 1:
        raise ValueError("world and align must be >= 1")
    nblk = -(-n_slow // align)
    if nblk < world:
        raise ValueError(f"{n_slow} planes make {nblk} blocks of {align}: fewer than {world} ranks")
    base, extra = divmod(nblk, world)
    slabs, b = [], 0
    for r in range(world):
        nb = base + (1 if r < extra else 0)
        lo, hi = b * align, min((b + nb) * align, n_slow)
        b += nb
        below = r - 1 if r > 0 else (world - 1 if periodic else None)
        above = r + 1 if r < world - 1 else (0 if periodic else None)
        slabs.append(Slab(r, lo, hi, below, above))
    return slabs


def crossing(q: int):
    """(up, down): populations that cross a cut going up (c = +1) and going down (c = -1)."""
    c = slab_velocity(q)
    return [i for i in range(q) if c[i] == 1], [i for i in range(q) if c[i] == -1]


def exchange_halos(f_ext, q: int, slab: Slab, group=None):
    """One halo exchange on a slab stored with a ghost plane on each side that has a neighbour:
    f_ext[q, planes..., rows, cells] along dim 1 (the slab axis), ghost planes first and last where
    present.  The populations moving up leave through the top owned plane into the upper
    neighbour's lower ghost plane, and those moving down through the bottom owned plane.  Sends
    only the crossing populations (contiguous copies), as point-to-point messages."""
    import torch
    import torch.distributed as dist

    up, down = crossing(q)
    lo_ghost = 1 if slab.below is not None else 0
    hi_ghost = 1 if slab.above is not None else 0
    first, last = lo_ghost, f_ext.shape[1] - 1 - hi_ghost  # owned planes
    reqs, recv = [], []
    if slab.above is not None:
        reqs.append(dist.isend(f_ext[up, last].contiguous(), slab.above, group=group, tag=1))
        buf = torch.empty_like(f_ext[down, f_ext.shape[1] - 1])
        reqs.append(dist.irecv(buf, slab.above, group=group, tag=2))
        recv.append((down, f_ext.shape[1] - 1, buf))
    if slab.below is not None:
        reqs.append(dist.isend(f_ext[down, first].contiguous(), slab.below, group=group, tag=2))
        buf = torch.empty_like(f_ext[up, 0])
        reqs.append(dist.irecv(buf, slab.below, group=group, tag=1))
        recv.append((up, 0, buf))
    for r in reqs:
        r.wait()
    for idx, plane, buf in recv:
        f_ext[idx, plane] = buf


def halo_faces(slab: Slab) -> int:
    """lbm_set_halo faces of a slab: the low face is cut where a rank lies below, the high face
    where one lies above."""
    from . import lbm as L

    return (L.LBM_HALO_LO if slab.below is not None else 0) | \
        (L.LBM_HALO_HI if slab.above is not None else 0)


def exchange_lattice_halos(lat, slab: Slab, group=None):
    """One halo exchange of a library slab (a `Lattice` whose cut faces have halos): the
    populations leaving through each cut face go to the neighbour across it, and the neighbour's go
    into the face's halo, through host memory as point-to-point messages of raw storage bytes
    (tag 1 travels up, tag 2 down, as in `exchange_halos`).  A slab that is its own neighbour (one
    rank, periodic slab axis) takes its own messages.  Call it between steps."""
    import torch
    import torch.distributed as dist

    from . import lbm as L

    me = dist.get_rank(group) if group is not None else dist.get_rank()
    out = {}
    if slab.above is not None:
        out["up"] = lat.halo_export(L.LBM_HALO_HI)
    if slab.below is not None:
        out["down"] = lat.halo_export(L.LBM_HALO_LO)
    reqs, recv = [], []
    if slab.above is not None:
        if slab.above == me:
            recv.append((L.LBM_HALO_HI, out["down"]))
        else:
            reqs.append(dist.isend(torch.from_numpy(out["up"]), slab.above, group=group, tag=1))
            buf = torch.empty(out["up"].size, dtype=torch.uint8)
            reqs.append(dist.irecv(buf, slab.above, group=group, tag=2))
            recv.append((L.LBM_HALO_HI, buf))
    if slab.below is not None:
        if slab.below == me:
            recv.append((L.LBM_HALO_LO, out["up"]))
        else:
            reqs.append(dist.isend(torch.from_numpy(out["down"]), slab.below, group=group, tag=2))
            buf = torch.empty(out["down"].size, dtype=torch.uint8)
            reqs.append(dist.irecv(buf, slab.below, group=group, tag=1))
            recv.append((L.LBM_HALO_LO, buf))
    for r in reqs:
        r.wait()
    for face, buf in recv:
        lat.halo_import(face, buf.numpy() if hasattr(buf, "numpy") else buf)


def gather_maxima(local, group=None):
    """All ranks' block maxima concatenated in rank order (slab order = global block order when
    the slab axis is the slowest one)."""
    import torch
    import torch.distributed as dist

    n = torch.tensor([local.numel()], dtype=torch.int64)
    sizes = [torch.zeros_like(n) for _ in range(dist.get_world_size(group))]
    dist.all_gather(sizes, n, group=group)
    m = int(max(s.item() for s in sizes))
    pad = torch.full((m,), float("nan"), dtype=local.dtype)
    pad[:local.numel()] = local.reshape(-1)
    parts = [torch.empty_like(pad) for _ in sizes]
    dist.all_gather(parts, pad, group=group)
    return torch.cat([p[:int(s.item())] for p, s in zip(parts, sizes)])


def allreduce_sums(sums, group=None):
    """Global mass and momentum from per-rank FP64 sums (in place)."""
    import torch.distributed as dist

    dist.all_reduce(sums, op=dist.ReduceOp.SUM, group=group)
    return sums
