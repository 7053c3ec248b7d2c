"""GPU parity of stencil_redblack_sweep (red-black Gauss-Seidel through the
sweep kernel with a colour mask per stage) against the CPU oracle's
in-place red-black sweeps."""
import numpy as np
import pytest

import oracle
from paper_2310_01882_b300 import stencil as S
from tests.gpu_util import ctx, halo_equal, rel_err

pytestmark = pytest.mark.gpu

SHAPES = [(64, 64, 64), (67, 35, 19), (1, 1, 1), (3, 130, 2), (130, 17, 70), (2, 2, 2)]


def rand_problem(nx, ny, nz, seed):
    rng = np.random.default_rng(seed)
    u = rng.random((nz + 2, ny + 2, nx + 2))  # nonzero Dirichlet halo
    f = rng.standard_normal((nz + 2, ny + 2, nx + 2))
    return u, f, 1.0 / (max(nx, ny, nz) + 1)


def rb(u_np, f_np, h, nsweeps, dtype=S.F64, flags=S.SWEEP_AUTO, spp=0, work=True):
    import torch
    u = S.Field.from_numpy(u_np, dtype)
    f = S.Field.from_numpy(f_np, dtype)
    w = S.Field(u.nx, u.ny, u.nz, S.F64) if work else None
    S.stencil_redblack_sweep(ctx(), u, u.like(), f, w, h, nsweeps, spp, flags)
    torch.cuda.synchronize()
    S.stencil_ctx_status(ctx())
    return u.to_numpy()


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("nsweeps", [1, 2, 3, 6])
@pytest.mark.parametrize("mode", ["resident", "per_pass", "native"])
def test_f64(shape, nsweeps, mode):
    """FP64: resident fixed point (work grid; from 2 sweeps on), fixed point
    per pass, binary64 arithmetic; 1e-13 against the oracle."""
    u, f, h = rand_problem(*shape, seed=sum(shape) + nsweeps)
    ref = oracle.rbgs(u, f, h, nsweeps)
    flags = S.SWEEP_FP64_NATIVE if mode == "native" else S.SWEEP_FP64_FIXED
    got = rb(u, f, h, nsweeps, flags=flags, work=(mode == "resident"))
    assert rel_err(got, ref) <= 1e-13
    assert halo_equal(got, u)


@pytest.mark.parametrize("shape", [(67, 35, 19), (130, 17, 70), (1, 1, 1), (5, 3, 2), (64, 64, 64)])
@pytest.mark.parametrize("nsweeps", [1, 2, 3, 5])
@pytest.mark.parametrize("spp", [1, 2])
def test_f32(shape, nsweeps, spp):
    """FP32 storage and arithmetic, one or two sweeps per pass, against the
    FP32 oracle from the same FP32-rounded input."""
    u, f, h = rand_problem(*shape, seed=50 + nsweeps)
    u32, f32 = u.astype(np.float32), f.astype(np.float32)
    ref = oracle.rbgs_f32(u32, f32, h, nsweeps).astype(np.float64)
    got = rb(u32.astype(np.float64), f32.astype(np.float64), h, nsweeps, dtype=S.F32, spp=spp)
    assert rel_err(got, ref) <= 1e-5 * nsweeps
    assert halo_equal(got, u32.astype(np.float64))


@pytest.mark.parametrize("shape", [(67, 35, 19), (130, 17, 70), (3, 2, 1)])
@pytest.mark.parametrize("nsweeps", [1, 2, 5])
@pytest.mark.parametrize("spp", [1, 2])
def test_bf16(shape, nsweeps, spp):
    """bf16 storage: one bf16 rounding per pass (the red values a pass
    computes stay binary32 for its black half), so the error against the
    FP64 sweeps of the same bf16-rounded input is at most 2^-8 per pass."""
    u, f, h = rand_problem(*shape, seed=70 + nsweeps)
    ub = oracle.from_bf16(oracle.to_bf16(u.astype(np.float32))).astype(np.float64)
    fb = oracle.from_bf16(oracle.to_bf16(f.astype(np.float32))).astype(np.float64)
    ref = oracle.rbgs(ub, fb, h, nsweeps)
    got = rb(ub, fb, h, nsweeps, dtype=S.BF16, spp=spp)
    passes = -(-nsweeps // spp)
    assert rel_err(got, ref) <= passes * 2.0 ** -8
    assert halo_equal(got, ub)


def test_differs_from_jacobi_and_converges_faster():
    """The colour mask is live: red-black is not two Jacobi sweeps, and it
    reaches the exact discrete solution faster."""
    from oracle import exact
    n = 24
    h = 1.0 / (n + 1)
    rng = np.random.default_rng(3)
    f = np.zeros((n + 2,) * 3)
    f[1:-1, 1:-1, 1:-1] = rng.standard_normal((n,) * 3)
    ud = exact.solve(f, h)
    z = np.zeros_like(f)
    got = rb(z, f, h, 40)
    assert rel_err(got, oracle.rbgs(z, f, h, 40)) <= 1e-13
    import torch
    u = S.Field.from_numpy(z)
    S.stencil_jacobi_sweep(ctx(), u, u.like(), S.Field.from_numpy(f), S.Field(n, n, n), h, 40)
    torch.cuda.synchronize()
    jac = u.to_numpy()
    # the smooth error decays like mu^(2k) against Jacobi's mu^k
    assert np.max(np.abs(got - ud)) < 0.8 * np.max(np.abs(jac - ud))


def test_arguments():
    u = S.Field(8, 8, 8)
    with pytest.raises(S.StencilError):
        S.stencil_redblack_sweep(ctx(), u, u.like(), u.like(), None, 0.1, 1, 5)  # sweeps_per_pass > 4
    with pytest.raises(S.StencilError):
        S.stencil_redblack_sweep(ctx(), u, u, u.like(), None, 0.1, 1, 0)  # u_tmp aliases u


RB_CONFIG_CASES = [(S.F64, S.SWEEP_FP64_FIXED, True, 1), (S.F64, S.SWEEP_FP64_FIXED, False, 1),
                   (S.F64, S.SWEEP_FP64_NATIVE, False, 1), (S.F32, 0, False, 1), (S.F32, 0, False, 2),
                   (S.BF16, 0, False, 1), (S.BF16, 0, False, 2)]


@pytest.mark.parametrize("dtype,flags,with_work,spp", RB_CONFIG_CASES)
@pytest.mark.parametrize("shape", [(70, 45, 23), (120, 40, 11)])
def test_every_compiled_configuration(dtype, flags, with_work, spp, shape):
    """Each compiled red-black tile configuration (pinned with
    redblack_config_select) gives the oracle's sweeps on a ragged grid and
    on one whose x extent fills whole 60-column tiles."""
    u, f, h = rand_problem(*shape, seed=43)
    n = 4
    if dtype == S.F64:
        u_in, f_in = u, f
        ref, tol = oracle.rbgs(u, f, h, n), 1e-13
    elif dtype == S.F32:
        u32, f32 = u.astype(np.float32), f.astype(np.float32)
        u_in, f_in = u32.astype(np.float64), f32.astype(np.float64)
        ref, tol = oracle.rbgs_f32(u32, f32, h, n).astype(np.float64), 1e-5 * n
    else:
        u_in = oracle.from_bf16(oracle.to_bf16(u.astype(np.float32))).astype(np.float64)
        f_in = oracle.from_bf16(oracle.to_bf16(f.astype(np.float32))).astype(np.float64)
        ref, tol = oracle.rbgs(u_in, f_in, h, n), (-(-n // spp)) * 2.0 ** -8
    c = S.Context(0)
    count = S.stencil_redblack_config_count(dtype, flags, with_work, spp)
    assert count >= 1
    for idx in range(count):
        S.stencil_redblack_config_select(c, dtype, flags, with_work, spp, idx)
        uf, ff = S.Field.from_numpy(u_in, dtype), S.Field.from_numpy(f_in, dtype)
        w = S.Field(uf.nx, uf.ny, uf.nz) if with_work else None
        S.stencil_redblack_sweep(c, uf, uf.like(), ff, w, h, n, spp, flags)
        S.stencil_ctx_status(c)
        got = uf.to_numpy()
        assert rel_err(got, ref) <= tol, (idx, rel_err(got, ref))
        assert halo_equal(got, u_in)
    with pytest.raises(S.StencilError):
        S.stencil_redblack_config_select(c, dtype, flags, with_work, spp, count)
    c.close()
