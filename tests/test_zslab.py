"""Z-slab decomposition with halo exchange (the paper's distributed-memory
path): the exchange schedule on CPU ranks (gloo, 2 and 3 processes, and
slabs in one process) with the oracle as each rank's sweep must reproduce
the whole-grid oracle sweeps bit for bit, one sweep per exchange or several
over a deeper halo; on one GPU, slabs as virtual ranks through the library
must match the oracle to 1e-13."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2310_01882_b300 import zslab


def test_slab_bounds_cover_the_grid():
    for nz, r in ((7, 3), (8, 2), (5, 5), (130, 4)):
        b = zslab.slab_bounds(nz, r)
        assert b[0][0] == 1 and b[-1][1] == nz + 1
        assert all(b[i][1] == b[i + 1][0] for i in range(r - 1))
        sizes = [z1 - z0 for z0, z1 in b]
        assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        zslab.slab_bounds(3, 4)


@pytest.mark.parametrize("depth", [1, 2, 3])
def test_split_join_roundtrip(depth):
    a = np.random.default_rng(0).random((11, 5, 6))
    slabs = zslab.split(a, 3, depth)
    assert np.array_equal(zslab.join(slabs, depth), a)
    # each slab holds its core plus `depth` ghost planes towards a neighbour
    # and the global halo plane at an end of the grid
    cores = [z1 - z0 for z0, z1 in zslab.slab_bounds(9, 3)]
    assert [s.shape[0] for s in slabs] == [cores[0] + 1 + depth, cores[1] + 2 * depth, cores[2] + depth + 1]
    with pytest.raises(ValueError):
        zslab.split(a, 3, 4)  # a ghost plane would come from two ranks away


@pytest.mark.parametrize("nranks,depth,nsweeps", [(2, 1, 4), (3, 2, 5), (4, 3, 7), (3, 3, 3)])
def test_local_exchange_reproduces_whole_grid(nranks, depth, nsweeps):
    """Slabs in one process (CPU tensors), the oracle as each slab's sweep:
    `depth` sweeps per exchange give the whole grid's sweeps bit for bit."""
    import torch
    u, f, h = _problem((6, 5, 13), seed=7)
    us = [torch.from_numpy(a) for a in zslab.split(u, nranks, depth)]
    fs = zslab.split(f, nranks, depth)
    ex = zslab.LocalExchange(us, depth)

    def make(t, fa):
        def sweep(n):
            t.copy_(torch.from_numpy(oracle.jacobi(t.numpy(), fa, h, n)))
        return sweep

    zslab.run([ex], [make(t, fa) for t, fa in zip(us, fs)], nsweeps, depth)
    got = zslab.join([t.numpy() for t in us], depth)
    assert np.array_equal(got, oracle.jacobi(u, f, h, nsweeps))


def _problem(shape, seed):
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    u = rng.random((nz + 2, ny + 2, nx + 2))
    f = rng.standard_normal(u.shape)
    return u, f, 1.0 / (max(shape) + 1)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, shape, nsweeps, depth, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    u, f, h = _problem(shape, seed=5)
    mine = torch.from_numpy(zslab.split(u, world, depth)[rank])
    f_mine = zslab.split(f, world, depth)[rank]
    ex = zslab.DistExchange(mine, rank, world, depth=depth)

    def sweep(n):
        for _ in range(n):
            mine.copy_(torch.from_numpy(oracle.jacobi_sweep(mine.numpy(), f_mine, h)))

    zslab.run([ex], [sweep], nsweeps, depth)
    q.put((rank, mine.numpy().copy()))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,shape,depth", [(2, (6, 5, 8), 1), (3, (5, 4, 7), 1), (3, (5, 4, 9), 3)])
def test_gloo_ranks_reproduce_whole_grid(world, shape, depth):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    nsweeps = 4
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, shape, nsweeps, depth, q))
             for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    u, f, h = _problem(shape, seed=5)
    ref = oracle.jacobi(u, f, h, nsweeps)
    assert np.array_equal(zslab.join([got[r] for r in range(world)], depth), ref)


@pytest.mark.gpu
@pytest.mark.parametrize("nslabs,shape,depth", [(3, (67, 35, 19), 1), (4, (32, 32, 64), 1), (2, (5, 3, 2), 1),
                                                (3, (67, 35, 19), 4), (4, (32, 32, 64), 8)])
def test_gpu_virtual_ranks(nslabs, shape, depth):
    import torch
    from paper_2310_01882_b300 import stencil as S
    from tests.gpu_util import rel_err
    u, f, h = _problem(shape, seed=9)
    nsweeps = 11
    ref = oracle.jacobi(u, f, h, nsweeps)
    for flags in (S.SWEEP_FP64_FIXED, S.SWEEP_FP64_NATIVE):
        fields, ex, fns = zslab.gpu_slabs(u, f, h, nslabs, flags=flags, depth=depth)
        zslab.run([ex], fns, nsweeps, depth)
        torch.cuda.synchronize()
        got = zslab.join([x.to_numpy() for x in fields], depth)
        assert rel_err(got, ref) <= 1e-13, flags
