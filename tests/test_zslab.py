"""Z-slab decomposition with halo exchange (the paper's distributed-memory
path): the exchange schedule on CPU ranks (gloo, 2 and 3 processes) with the
oracle as each rank's sweep must reproduce the whole-grid oracle sweeps bit
for bit; on one GPU, slabs as virtual ranks through the library must match
the oracle to 1e-13."""
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


def test_split_join_roundtrip():
    a = np.random.default_rng(0).random((9, 5, 6))
    assert np.array_equal(zslab.join(zslab.split(a, 3)), a)


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


def _rank_main(rank, world, port, shape, nsweeps, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    u, f, h = _problem(shape, seed=5)
    mine = torch.from_numpy(zslab.split(u, world)[rank])
    f_mine = zslab.split(f, world)[rank]
    ex = zslab.DistExchange(mine, rank, world)

    def sweep():
        mine.copy_(torch.from_numpy(oracle.jacobi_sweep(mine.numpy(), f_mine, h)))

    zslab.run([ex], [sweep], nsweeps)
    q.put((rank, mine.numpy().copy()))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,shape", [(2, (6, 5, 8)), (3, (5, 4, 7))])
def test_gloo_ranks_reproduce_whole_grid(world, shape):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    nsweeps = 4
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, shape, nsweeps, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(120)
    assert all(p.exitcode == 0 for p in procs)
    u, f, h = _problem(shape, seed=5)
    ref = oracle.jacobi(u, f, h, nsweeps)
    assert np.array_equal(zslab.join([got[r] for r in range(world)]), ref)


@pytest.mark.gpu
@pytest.mark.parametrize("nslabs,shape", [(3, (67, 35, 19)), (4, (32, 32, 64)), (2, (5, 3, 2))])
def test_gpu_virtual_ranks(nslabs, shape):
    import torch
    from paper_2310_01882_b300 import stencil as S
    from tests.gpu_util import rel_err
    u, f, h = _problem(shape, seed=9)
    for flags in (S.SWEEP_FP64_FIXED, S.SWEEP_FP64_NATIVE):
        fields, ex, fns = zslab.gpu_slabs(u, f, h, nslabs, flags=flags)
        zslab.run([ex], fns, 5)
        torch.cuda.synchronize()
        got = zslab.join([x.to_numpy() for x in fields])
        ref = oracle.jacobi(u, f, h, 5)
        assert rel_err(got, ref) <= 1e-13, flags
