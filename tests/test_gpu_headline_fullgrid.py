"""Full-grid parity of the throughput workload in the benchmark's own launch
configuration: 512^3, h = 1/513, source a k^-3 Gaussian random field (seed
2), start U[0,1) (seed 3), zero Dirichlet halo; the sweep configuration the
autotuner keeps for these grids, one sweep per pass, the work grid given.
Every interior point is compared with the binary64 oracle after 1, 2 and 8
sweeps (the loop oracle, chained), and after 1000 sweeps -- one benchmark
step -- with the oracle's closed form of the sweeps (oracle/exact.py), at the
FP64 tolerance 1e-13."""
import numpy as np
import pytest

import oracle
from oracle import exact
from paper_2310_01882_b300 import inputs
from paper_2310_01882_b300 import stencil as S
from tests.gpu_util import ctx, halo_equal, rel_err

pytestmark = pytest.mark.gpu

N = 512
TOL = 1e-13


def test_headline_512cubed_every_point():
    import torch
    f = inputs.grf(N, seed=2)
    u0 = inputs.uniform(N, N, N, seed=3)
    h = 1.0 / (N + 1)
    c = ctx()
    u, ut, fd = S.Field.from_numpy(u0), S.Field(N, N, N), S.Field.from_numpy(f)
    work = S.Field(N, N, N)
    u0_dev = torch.from_numpy(u0).cuda()
    S.stencil_autotune_sweep(c, u, ut, fd, work, h)

    def run(nsweeps):
        u.cells.copy_(u0_dev)
        S.stencil_jacobi_sweep(c, u, ut, fd, work, h, nsweeps, 1, S.SWEEP_AUTO)
        torch.cuda.synchronize()
        S.stencil_ctx_status(c)
        return u.to_numpy()

    ref = u0
    done = 0
    for n in (1, 2, 8):
        ref = oracle.jacobi(ref, f, h, n - done, nthreads=0)
        done = n
        got = run(n)
        assert rel_err(got, ref) <= TOL, (n, rel_err(got, ref))
        assert halo_equal(got, u0)
    got = run(1000)
    ref = exact.jacobi_sweeps(u0, f, h, 1000)
    assert rel_err(got, ref) <= TOL, (1000, rel_err(got, ref))
    assert halo_equal(got, u0)
