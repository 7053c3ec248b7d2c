"""Z-slab domain decomposition of the Jacobi sweep with a halo exchange.

The paper's distributed-memory path splits the grid across processes and
swaps halos every iteration (Sections 3 and 4.2).  Here the z range of one
grid is cut into contiguous slabs, one per rank; every slab is an ordinary
grid (its own one-cell halo) whose two z halo planes hold the neighbouring
slabs' boundary planes (or the global Dirichlet planes at the ends).  One
step = exchange those planes, then one sweep of every slab through the
library (stencil_jacobi_sweep), so the slabs together reproduce the sweep of
the whole grid point for point.

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
    """Interior planes [z0, z1) (1-based halo indices) of each rank's slab:
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


def split(a, nranks):
    """Cut a halo field (..., nz+2, ny+2, nx+2 along the first axis = z) into
    per-rank slab arrays with their own z halo planes (copies)."""
    nz = a.shape[0] - 2
    return [a[z0 - 1:z1 + 1].copy() if hasattr(a, "copy") else a[z0 - 1:z1 + 1].clone()
            for z0, z1 in slab_bounds(nz, nranks)]


def join(slabs):
    """Reassemble slab arrays (numpy) into the whole halo field."""
    import numpy as np
    parts = [slabs[0][:1]] + [s[1:-1] for s in slabs] + [slabs[-1][-1:]]
    return np.concatenate(parts, axis=0)


class LocalExchange:
    """All slabs in this process: plane copies between the slabs' tensors
    (`planes[r]` is a (nz_r + 2, ny + 2, nx + 2)-shaped tensor view of slab
    r's cells)."""

    def __init__(self, planes):
        self.planes = planes

    def exchange(self):
        p = self.planes
        for r in range(len(p) - 1):
            p[r + 1][0].copy_(p[r][-2])   # my top interior plane -> next slab's bottom halo
            p[r][-1].copy_(p[r + 1][1])   # next slab's bottom interior plane -> my top halo


class DistExchange:
    """One slab per process (rank r of `world`): the boundary planes go to
    the neighbouring ranks with torch.distributed send/recv."""

    def __init__(self, plane_view, rank, world, group=None):
        self.p, self.rank, self.world, self.group = plane_view, rank, world, group

    def exchange(self):
        import torch.distributed as dist
        p, r = self.p, self.rank
        ops = []
        if r + 1 < self.world:
            ops.append(dist.P2POp(dist.isend, p[-2].contiguous(), r + 1, self.group))
            top = p[-1].clone()
            ops.append(dist.P2POp(dist.irecv, top, r + 1, self.group))
        if r > 0:
            ops.append(dist.P2POp(dist.isend, p[1].contiguous(), r - 1, self.group))
            bottom = p[0].clone()
            ops.append(dist.P2POp(dist.irecv, bottom, r - 1, self.group))
        if ops:
            for req in dist.batch_isend_irecv(ops):
                req.wait()
        if r + 1 < self.world:
            p[-1].copy_(top)
        if r > 0:
            p[0].copy_(bottom)


def run(exchanges, sweep_fns, nsweeps):
    """nsweeps steps: every transport exchanges its halo planes, then every
    slab is swept once.  `exchanges`: objects with .exchange(); `sweep_fns`:
    one callable per local slab (one sweep in place)."""
    for _ in range(nsweeps):
        for ex in exchanges:
            ex.exchange()
        for fn in sweep_fns:
            fn()


def gpu_slabs(u_np, f_np, h, nslabs, dtype=None, flags=None, ctx=None):
    """Virtual ranks on one GPU: the grid's slabs as library Fields, a
    LocalExchange over them and one sweep callable per slab
    (stencil_jacobi_sweep, one sweep, no work grid).  Returns
    (fields, exchange, sweep_fns)."""
    from . import stencil as S
    dtype = S.F64 if dtype is None else dtype
    flags = S.SWEEP_AUTO if flags is None else flags
    ctx = ctx or S.Context(0)
    us = [S.Field.from_numpy(a, dtype) for a in split(u_np, nslabs)]
    fs = [S.Field.from_numpy(a, dtype) for a in split(f_np, nslabs)]
    tmps = [u.like() for u in us]
    ex = LocalExchange([u.cells for u in us])
    fns = [(lambda u=u, t=t, f=f: S.stencil_jacobi_sweep(ctx, u, t, f, None, h, 1, 1, flags))
           for u, t, f in zip(us, tmps, fs)]
    return us, ex, fns
