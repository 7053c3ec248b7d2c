"""FP64 sweeps on inputs whose solution is far below any a-priori bound on
the iterates: zero start with a checkerboard source, a single-cell point
source, and a source of 1e-12 beside a Dirichlet halo of 1, over thousands of
sweeps, through the library's default FP64 arithmetic (STENCIL_SWEEP_AUTO:
fixed point with a per-pass scale), with and without a work grid, for
Jacobi, red-black Gauss-Seidel and the z-slab decomposition; element by
element over the whole grid against the binary64 oracle at 1e-13.  Also:
the kernel's integers equal the host model of its arithmetic
(tests/fixed_point_model.py) bit for bit."""
import numpy as np
import pytest

import oracle
from paper_2310_01882_b300 import stencil as S
from paper_2310_01882_b300 import zslab
from tests import fixed_point_model as FX
from tests.gpu_util import ctx, halo_equal, rel_err, sweep
from tests.test_fixed_point_model import hard_inputs

pytestmark = pytest.mark.gpu

TOL = 1e-13
CASES = [(64, 5000), (128, 2000)]
NAMES = ["checkerboard", "point", "tiny_source_halo_1"]

_refs = {}


def reference(kind, n, nsweeps, name):
    key = (kind, n, nsweeps, name)
    if key not in _refs:
        h, cs = hard_inputs(n)
        u0, f = cs[name]
        run = oracle.jacobi if kind == "jacobi" else oracle.rbgs
        _refs[key] = (u0, f, h, run(u0, f, h, nsweeps, nthreads=0))
    return _refs[key]


def redblack(u_np, f_np, h, nsweeps, work):
    import torch
    u = S.Field.from_numpy(u_np)
    f = S.Field.from_numpy(f_np)
    w = S.Field(u.nx, u.ny, u.nz, S.F64) if work else None
    S.stencil_redblack_sweep(ctx(), u, u.like(), f, w, h, nsweeps, 0, S.SWEEP_AUTO)
    torch.cuda.synchronize()
    S.stencil_ctx_status(ctx())
    return u.to_numpy()


@pytest.mark.parametrize("n,nsweeps", CASES)
@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("work", [True, False], ids=["resident", "per_pass"])
def test_jacobi(n, nsweeps, name, work):
    u0, f, h, ref = reference("jacobi", n, nsweeps, name)
    got = sweep(u0, f, h, nsweeps, flags=S.SWEEP_AUTO, work=work)
    assert rel_err(got, ref) <= TOL, (name, rel_err(got, ref))
    assert halo_equal(got, u0)


@pytest.mark.parametrize("n,nsweeps", CASES)
@pytest.mark.parametrize("name", NAMES)
def test_jacobi_two_sweeps_per_pass(n, nsweeps, name):
    u0, f, h, ref = reference("jacobi", n, nsweeps, name)
    got = sweep(u0, f, h, nsweeps, flags=S.SWEEP_AUTO, spp=2, work=True)
    assert rel_err(got, ref) <= TOL, (name, rel_err(got, ref))


@pytest.mark.parametrize("n,nsweeps", CASES)
@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("work", [True, False], ids=["resident", "per_pass"])
def test_redblack(n, nsweeps, name, work):
    u0, f, h, ref = reference("redblack", n, nsweeps, name)
    got = redblack(u0, f, h, nsweeps, work)
    assert rel_err(got, ref) <= TOL, (name, rel_err(got, ref))
    assert halo_equal(got, u0)


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("depth", [1, 8])
def test_zslab(name, depth):
    """Four virtual ranks on one GPU, a halo exchange every `depth` sweeps."""
    import torch
    n, nsweeps = 64, 2000
    u0, f, h, ref = reference("jacobi", n, nsweeps, name)
    fields, ex, fns = zslab.gpu_slabs(u0, f, h, 4, flags=S.SWEEP_AUTO, ctx=ctx(), depth=depth)
    zslab.run([ex], fns, nsweeps, depth)
    torch.cuda.synchronize()
    got = zslab.join([x.to_numpy() for x in fields], depth)
    assert rel_err(got, ref) <= TOL, (name, depth, rel_err(got, ref))


@pytest.mark.parametrize("T", [1, 2])
@pytest.mark.parametrize("name", ["checkerboard", "random"])
def test_kernel_equals_model(T, name):
    """The resident fixed-point sweep's result equals, bit for bit, the host
    model of its integer arithmetic (scale per pass, rescaling, source
    shift, rounding), on a ragged grid with a nonzero halo."""
    nx, ny, nz = 45, 33, 29
    rng = np.random.default_rng(17 + T)
    u0 = np.zeros((nz + 2, ny + 2, nx + 2))
    f = np.zeros_like(u0)
    if name == "checkerboard":
        k, j, i = np.meshgrid(np.arange(nz + 2), np.arange(ny + 2), np.arange(nx + 2), indexing="ij")
        f[FX.I3] = np.where((i + j + k) % 2 == 0, 1.0, -1.0)[FX.I3]
        u0[0] = rng.random(u0[0].shape) * 1e-3
    else:
        u0[:] = rng.random(u0.shape)
        f[FX.I3] = rng.standard_normal((nz, ny, nx))
    h = 1.0 / 46
    nsweeps = 60
    got = sweep(u0, f, h, nsweeps, flags=S.SWEEP_FP64_FIXED, spp=T, work=True)
    want = FX.pass_scale(u0, f, h, nsweeps, T=T)
    assert np.array_equal(got.view(np.int64), want.view(np.int64))
