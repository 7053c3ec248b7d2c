"""Z-slab domain decomposition of the Jacobi sweep with a halo exchange.

The paper's distributed-memory path splits the grid across processes and
swaps halos every iteration (Sections 3 and 4.2).  Here the z range of one
grid is cut into contiguous slabs, one per rank.  Every slab is an ordinary
grid (its own one-cell halo) made of the rank's core planes plus `depth`
ghost planes on each side that faces another slab (the outermost of them is
the slab's halo plane; at the two ends of the grid the slab's halo is the
global Dirichlet plane).  One step = exchange the ghost planes (each rank
sends the `depth` core planes next to each neighbour), then `depth` sweeps
of every slab through the library (stencil_jacobi_sweep).  A ghost plane
that the slab sweeps goes stale by one plane per sweep from the slab's
edge, so after `depth` sweeps exactly the core planes are right and the
slabs together reproduce the sweeps of the whole grid point for point;
depth 1 is the paper's swap per iteration, a deeper halo trades redundant
ghost-plane sweeps for fewer exchanges (and lets the library fuse sweeps).

Two transports share the same exchange schedule:
  * `DistExchange`: one slab per process, planes sent with
    torch.distributed point-to-point calls (NCCL between GPUs, gloo on CPU);
  * `LocalExchange`: every slab in one process (virtual ranks on one GPU),
    planes copied between the slabs' buffers in stream order.
The sweep itself is a callable, so the host logic can be driven on CPU with
any per-slab sweep.  Host orchestration only: the arithmetic runs in the
library's kernels (or in the caller's sweep function).
"""


def slab_bounds(nz, nranks):
    """Interior planes [z0, z1) (1-based halo indices) of each rank's core:
    as even as possible, the first nz % nranks slabs one plane thicker."""
    if not 1 <= nranks <= nz:
        raise ValueError(f"need 1 <= ranks <= nz (got {nranks} ranks for {nz} planes)")
    base, extra = divmod(nz, nranks)
    out, z = [], 1
    for r in range(nranks):
        n = base + (1 if r < extra else 0)
        out.append((z, z + n))
        z += n
    return out


def ghosts(rank, nranks, depth=1):
    """(planes below, planes above) the core of rank's slab array: the
    global halo plane (1) at an end of the grid, `depth` ghost planes
    towards a neighbour."""
    return (1 if rank == 0 else depth), (1 if rank == nranks - 1 else depth)


def slab_extent(nz, nranks, rank, depth=1):
    """Global planes [lo, hi] (inclusive, 0 and nz+1 are the halo) that
    rank's slab array holds."""
    z0, z1 = slab_bounds(nz, nranks)[rank]
    below, above = ghosts(rank, nranks, depth)
    return z0 - below, z1 - 1 + above


def check_depth(nz, nranks, depth):
    """Every ghost plane must come from the adjacent rank's core."""
    if depth < 1:
        raise ValueError(f"halo depth must be >= 1 (got {depth})")
    if nranks > 1 and min(z1 - z0 for z0, z1 in slab_bounds(nz, nranks)) < depth:
        raise ValueError(f"halo depth {depth} exceeds the thinnest core of {nz} planes over {nranks} ranks")


def split(a, nranks, depth=1):
    """Cut a halo field (..., nz+2, ny+2, nx+2 along the first axis = z) into
    per-rank slab arrays with their ghost and halo planes (copies)."""
    nz = a.shape[0] - 2
    check_depth(nz, nranks, depth)
    out = []
    for r in range(nranks):
        lo, hi = slab_extent(nz, nranks, r, depth)
        out.append(a[lo:hi + 1].copy() if hasattr(a, "copy") else a[lo:hi + 1].clone())
    return out


def join(slabs, depth=1):
    """Reassemble slab arrays (numpy) into the whole halo field: the global
    halo planes of the end slabs and every slab's core."""
    import numpy as np
    n = len(slabs)
    parts = [slabs[0][:1]]
    for r, s in enumerate(slabs):
        below, above = ghosts(r, n, depth)
        parts.append(s[below:s.shape[0] - above])
    parts.append(slabs[-1][-1:])
    return np.concatenate(parts, axis=0)


class LocalExchange:
    """All slabs in this process: plane copies between the slabs' tensors
    (`planes[r]` is a tensor view of slab r's cells, z first)."""

    def __init__(self, planes, depth=1):
        self.planes, self.depth = planes, depth

    def exchange(self):
        p, d, n = self.planes, self.depth, len(self.planes)
        for r in range(n - 1):
            above = ghosts(r, n, d)[1]
            below_next = ghosts(r + 1, n, d)[0]
            top = p[r].shape[0] - above         # end of slab r's core
            # slab r's top core planes -> slab r+1's lower ghosts, and slab
            # r+1's bottom core planes -> slab r's upper ghosts
            p[r + 1][0:d].copy_(p[r][top - d:top])
            p[r][top:top + d].copy_(p[r + 1][below_next:below_next + d])


class DistExchange:
    """One slab per process (rank r of `world`): the `depth` core planes next
    to each neighbour go to it with torch.distributed send/recv."""

    def __init__(self, plane_view, rank, world, group=None, depth=1):
        self.p, self.rank, self.world, self.group, self.depth = plane_view, rank, world, group, depth

    def exchange(self):
        import torch.distributed as dist
        p, r, d = self.p, self.rank, self.depth
        below, above = ghosts(r, self.world, d)
        top = p.shape[0] - above                 # end of my core
        ops = []
        if r + 1 < self.world:
            ops.append(dist.P2POp(dist.isend, p[top - d:top].contiguous(), r + 1, self.group))
            upper = p[top:top + d].clone()
            ops.append(dist.P2POp(dist.irecv, upper, r + 1, self.group))
        if r > 0:
            ops.append(dist.P2POp(dist.isend, p[below:below + d].contiguous(), r - 1, self.group))
            lower = p[0:d].clone()
            ops.append(dist.P2POp(dist.irecv, lower, r - 1, self.group))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()
        if r + 1 < self.world:
            p[top:top + d].copy_(upper)
        if r > 0:
            p[0:d].copy_(lower)


def run(exchanges, sweep_fns, nsweeps, depth=1):
    """nsweeps sweeps in steps of at most `depth`: every transport exchanges
    its ghost planes, then every slab is swept.  `exchanges`: objects with
    .exchange(); `sweep_fns`: one callable per local slab, called with the
    number of sweeps to apply in place."""
    left = nsweeps
    while left > 0:
        s = min(depth, left)
        for ex in exchanges:
            ex.exchange()
        for fn in sweep_fns:
            fn(s)
        left -= s


def gpu_slabs(u_np, f_np, h, nslabs, dtype=None, flags=None, ctx=None, depth=1):
    """Virtual ranks on one GPU: the grid's slabs as library Fields, a
    LocalExchange over them and one sweep callable per slab
    (stencil_jacobi_sweep of the requested sweeps, the library's pass
    length; FP64 slabs get a work grid, so from 4 sweeps on the iterate stays
    in fixed point for the call).  Returns (fields, exchange, sweep_fns)."""
    from . import stencil as S
    dtype = S.F64 if dtype is None else dtype
    flags = S.SWEEP_AUTO if flags is None else flags
    ctx = ctx or S.Context(0)
    us = [S.Field.from_numpy(a, dtype) for a in split(u_np, nslabs, depth)]
    fs = [S.Field.from_numpy(a, dtype) for a in split(f_np, nslabs, depth)]
    tmps = [u.like() for u in us]
    works = [S.Field(u.nx, u.ny, u.nz) if dtype == S.F64 else None for u in us]
    ex = LocalExchange([u.cells for u in us], depth)
    fns = [(lambda n, u=u, t=t, f=f, w=w: S.stencil_jacobi_sweep(ctx, u, t, f, w, h, n, 0, flags))
           for u, t, f, w in zip(us, tmps, fs, works)]
    return us, ex, fns
