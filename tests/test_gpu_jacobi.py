"""GPU parity of stencil_jacobi_sweep against the CPU oracle."""
import numpy as np
import pytest

import oracle
from paper_2310_01882_b300 import inputs
from paper_2310_01882_b300 import stencil as S
from tests.gpu_util import ctx, halo_equal, rel_err, sweep

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-13
FP32_TOL = 1e-5
BF16_TOL = 2.0 ** -7

SHAPES = [(64, 64, 64), (67, 35, 19), (1, 1, 1), (3, 130, 2), (130, 17, 70), (200, 48, 9)]


def rand_problem(nx, ny, nz, seed, halo=True):
    rng = np.random.default_rng(seed)
    u = rng.random((nz + 2, ny + 2, nx + 2))
    if not halo:
        u[0], u[-1], u[:, 0], u[:, -1], u[:, :, 0], u[:, :, -1] = 0, 0, 0, 0, 0, 0
    f = rng.standard_normal((nz + 2, ny + 2, nx + 2))
    return u, f, 1.0 / (max(nx, ny, nz) + 1)


def test_config0_64cubed_100_sweeps():
    """64^3, h = 1/65, f = 3 pi^2 sin sin sin, u0 ~ U[0,1) seed 1, 100 sweeps."""
    f, h = inputs.sin_source(64)
    u0 = inputs.uniform(64, 64, 64, seed=1)
    ref = oracle.jacobi(u0, f, h, 100, nthreads=0)
    for flags, work in ((S.SWEEP_FP64_FIXED, True), (S.SWEEP_FP64_FIXED, False), (S.SWEEP_FP64_NATIVE, False)):
        got = sweep(u0, f, h, 100, flags=flags, work=work)
        assert rel_err(got, ref) <= FP64_TOL, (flags, work)
        assert halo_equal(got, u0)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("nsweeps", [1, 2, 3, 4, 7])
@pytest.mark.parametrize("mode", ["resident", "per_pass", "native"])
def test_f64_ragged(shape, nsweeps, mode):
    """FP64: fixed point resident for the call (work grid), fixed point
    converted every pass (no work grid), and binary64 arithmetic; random
    nonzero Dirichlet halo."""
    u, f, h = rand_problem(*shape, seed=hash((shape, nsweeps)) % 1000)
    ref = oracle.jacobi(u, f, h, nsweeps)
    flags = S.SWEEP_FP64_NATIVE if mode == "native" else S.SWEEP_FP64_FIXED
    got = sweep(u, f, h, nsweeps, flags=flags, work=(mode == "resident"))
    assert rel_err(got, ref) <= FP64_TOL
    assert halo_equal(got, u)


def test_f64_halo_bits_preserved_with_awkward_values():
    """Dirichlet values with full 53-bit significands far below the fixed-point
    resolution (and a negative zero) come back bit for bit."""
    u, f, h = rand_problem(20, 11, 9, seed=5)
    rng = np.random.default_rng(6)
    u[0] = rng.standard_normal(u[0].shape) * 1e-30
    u[:, 0] = np.pi * 1e-20
    u[:, :, -1] = -0.0
    for mode in ("resident", "per_pass"):
        got = sweep(u, f, h, 6, flags=S.SWEEP_FP64_FIXED, work=(mode == "resident"))
        m = np.ones(u.shape, dtype=bool)
        m[1:-1, 1:-1, 1:-1] = False
        assert np.array_equal(got[m].view(np.int64), u[m].view(np.int64)), mode
        assert rel_err(got, oracle.jacobi(u, f, h, 6)) <= FP64_TOL


@pytest.mark.parametrize("shape", [(67, 35, 19), (130, 17, 70), (1, 1, 1), (5, 3, 2)])
@pytest.mark.parametrize("nsweeps", [1, 2, 3, 5, 8])
@pytest.mark.parametrize("spp", [1, 2])
def test_fixed_temporal_blocking(shape, nsweeps, spp):
    """Sweeps fused into one pass (T = 2, resident fixed point) equal
    separate sweeps to 1e-13."""
    u, f, h = rand_problem(*shape, seed=11 + nsweeps)
    ref = oracle.jacobi(u, f, h, nsweeps)
    got = sweep(u, f, h, nsweeps, flags=S.SWEEP_FP64_FIXED, spp=spp)
    assert rel_err(got, ref) <= FP64_TOL
    assert halo_equal(got, u)


@pytest.mark.parametrize("shape", [(67, 35, 19), (130, 17, 70), (1, 1, 1), (5, 3, 2), (64, 64, 64)])
@pytest.mark.parametrize("nsweeps", [1, 2, 3, 5, 8])
@pytest.mark.parametrize("spp", [1, 2, 4])
def test_f32_temporal_blocking(shape, nsweeps, spp):
    """FP32 passes of spp sweeps against the FP32-arithmetic oracle run sweep
    by sweep (the kernel keeps intermediate sweeps in binary32 registers,
    which is what binary32 storage holds)."""
    u, f, h = rand_problem(*shape, seed=21 + nsweeps)
    a = u.astype(np.float32)
    fb = f.astype(np.float32)
    for _ in range(nsweeps):
        a = oracle.jacobi_sweep_f32(a, fb, h)
    got = sweep(u.astype(np.float32).astype(np.float64), fb.astype(np.float64), h, nsweeps, dtype=S.F32, spp=spp)
    assert rel_err(got, a.astype(np.float64)) <= FP32_TOL
    assert halo_equal(got, u.astype(np.float32).astype(np.float64))


@pytest.mark.parametrize("shape", [(67, 35, 19), (130, 17, 70), (3, 2, 1)])
@pytest.mark.parametrize("nsweeps", [1, 2, 5, 8])
@pytest.mark.parametrize("spp", [1, 2, 4])
def test_bf16_temporal_blocking(shape, nsweeps, spp):
    """BF16 storage: each pass rounds once to bfloat16 (intermediate sweeps of
    a pass stay binary32), so the error against the FP64 sweeps of the same
    bf16-rounded input is at most one bf16 rounding (2^-8 relative) per pass."""
    u, f, h = rand_problem(*shape, seed=31 + nsweeps)
    ub = oracle.from_bf16(oracle.to_bf16(u.astype(np.float32))).astype(np.float64)
    fb = oracle.from_bf16(oracle.to_bf16(f.astype(np.float32))).astype(np.float64)
    ref = oracle.jacobi(ub, fb, h, nsweeps)
    got = sweep(ub, fb, h, nsweeps, dtype=S.BF16, spp=spp)
    passes = -(-nsweeps // spp)
    assert rel_err(got, ref) <= passes * 2.0 ** -8
    assert halo_equal(got, ub)


@pytest.mark.parametrize("shape", SHAPES)
def test_f32_per_sweep(shape):
    u, f, h = rand_problem(*shape, seed=7)
    u32, f32 = u.astype(np.float32), f.astype(np.float32)
    ref = oracle.jacobi_sweep(u32.astype(np.float64), f32.astype(np.float64),
                              float(np.sqrt(np.float64(oracle.f32_coeff(h)))))
    got = sweep(u32.astype(np.float64), f32.astype(np.float64), h, 1, dtype=S.F32)
    assert rel_err(got, ref) <= FP32_TOL
    assert halo_equal(got, u32.astype(np.float64))


@pytest.mark.parametrize("shape", SHAPES)
def test_bf16_per_sweep(shape):
    u, f, h = rand_problem(*shape, seed=8)
    ub = oracle.from_bf16(oracle.to_bf16(u.astype(np.float32))).astype(np.float64)
    fb = oracle.from_bf16(oracle.to_bf16(f.astype(np.float32))).astype(np.float64)
    ref = oracle.jacobi_sweep(ub, fb, h)
    got = sweep(ub, fb, h, 1, dtype=S.BF16)
    assert rel_err(got, ref) <= BF16_TOL
    assert halo_equal(got, ub)


def test_f32_multi_sweep_vs_f32_oracle():
    """20 FP32 sweeps against the FP32-arithmetic oracle (same storage
    rounding each sweep); the operation order differs only by one fused
    multiply-add and the reciprocal multiply."""
    u, f, h = rand_problem(70, 33, 21, seed=9)
    a = u.astype(np.float32)
    fb = f.astype(np.float32)
    for _ in range(20):
        a = oracle.jacobi_sweep_f32(a, fb, h)
    got = sweep(u.astype(np.float32).astype(np.float64), fb.astype(np.float64), h, 20, dtype=S.F32)
    assert rel_err(got, a.astype(np.float64)) <= FP32_TOL


def test_zero_sweeps_is_noop():
    u, f, h = rand_problem(9, 9, 9, seed=3)
    got = sweep(u, f, h, 0)
    assert np.array_equal(got, u)


def test_mode_decay_1000_sweeps_512():
    """Full-size property check (512^3, the benchmark launch configuration):
    with f = 0 the sine mode (1,2,3) decays by exactly mu^1000."""
    n = 512
    i = np.arange(n + 2, dtype=np.float64)
    sx = np.sin(np.pi * i / (n + 1)); sx[0] = sx[-1] = 0
    sy = np.sin(2 * np.pi * i / (n + 1)); sy[0] = sy[-1] = 0
    sz = np.sin(3 * np.pi * i / (n + 1)); sz[0] = sz[-1] = 0
    e0 = sz[:, None, None] * sy[None, :, None] * sx[None, None, :]
    mu = (np.cos(np.pi / (n + 1)) + np.cos(2 * np.pi / (n + 1)) + np.cos(3 * np.pi / (n + 1))) / 3
    got = sweep(e0, np.zeros_like(e0), 1.0 / (n + 1), 1000)
    assert rel_err(got, mu ** 1000 * e0) <= FP64_TOL


def test_full_size_sampled_one_sweep():
    """512^3 FP64 (k^-3 random field source, U[0,1) start): one sweep, and
    1000 further sweeps of the same launch configuration; sampled outputs
    of the first sweep are recomputed one by one from the definition's
    oracle (7 values each)."""
    n = 512
    f = inputs.grf(n, seed=2)
    u0 = inputs.uniform(n, n, n, seed=3)
    h = 1.0 / (n + 1)
    got = sweep(u0, f, h, 1)
    rng = np.random.default_rng(0)
    pts = rng.integers(1, n + 1, size=(2000, 3))
    pts = np.vstack([pts, [[1, 1, 1], [n, n, n], [1, n, 1], [n, 1, n]]])
    for (i, j, k) in pts:
        sub_u = u0[k - 1:k + 2, j - 1:j + 2, i - 1:i + 2]
        sub_f = f[k - 1:k + 2, j - 1:j + 2, i - 1:i + 2]
        ref = oracle.jacobi_sweep(sub_u, sub_f, h)[1, 1, 1]
        assert abs(got[k, j, i] - ref) <= FP64_TOL * max(1.0, abs(ref))


def test_fixed_nonfinite_input_reports():
    u, f, h = rand_problem(10, 10, 10, seed=4)
    f[5, 5, 5] = np.nan
    for nsw, work in ((2, None), (6, S.Field(10, 10, 10))):
        uf = S.Field.from_numpy(u)
        ff = S.Field.from_numpy(f)
        t = uf.like()
        S.stencil_jacobi_sweep(ctx(), uf, t, ff, work, h, nsw, 0, S.SWEEP_FP64_FIXED)
        with pytest.raises(S.StencilError) as e:
            S.stencil_ctx_status(ctx())
        assert e.value.code == -6
        out = uf.to_numpy()
        assert np.all(np.isnan(out[1:-1, 1:-1, 1:-1]))
        S.stencil_ctx_status(ctx())  # cleared


def test_argument_errors():
    u = S.Field(8, 8, 8)
    f = S.Field(8, 8, 8)
    with pytest.raises(S.StencilError) as e:
        S.stencil_jacobi_sweep(ctx(), u, u, f, None, 0.1, 1)
    assert e.value.code == -1
    t = S.Field(8, 8, 9)
    with pytest.raises(S.StencilError) as e:
        S.stencil_jacobi_sweep(ctx(), u, t, f, None, 0.1, 1)
    assert e.value.code == -1
    t = S.Field(8, 8, 8, S.F32)
    with pytest.raises(S.StencilError) as e:
        S.stencil_jacobi_sweep(ctx(), u, t, f, None, 0.1, 1)
    assert e.value.code == -3
    with pytest.raises(S.StencilError) as e:
        S.stencil_jacobi_sweep(ctx(), u, S.Field(8, 8, 8), f, S.Field(8, 8, 8, S.F32), 0.1, 5)
    assert e.value.code == -3
    # misaligned data pointer: shift the view by one element
    t = S.Field(8, 8, 8)
    g = t.grid()
    g.data = g.data + 8
    import ctypes
    gu, gf = u.grid(), f.grid()
    rc = S.lib().stencil_jacobi_sweep(ctx().handle, ctypes.byref(gu), ctypes.byref(g), ctypes.byref(gf),
                                      None, 0.1, 1, 0, 0, None)
    assert rc == -2


CONFIG_CASES = [(S.F64, S.SWEEP_FP64_FIXED, True), (S.F64, S.SWEEP_FP64_FIXED, False),
                (S.F64, S.SWEEP_FP64_NATIVE, False), (S.F32, 0, False), (S.BF16, 0, False)]


@pytest.mark.parametrize("dtype,flags,with_work", CONFIG_CASES)
@pytest.mark.parametrize("shape", [(70, 45, 23), (96, 40, 11)])
def test_every_compiled_configuration(dtype, flags, with_work, shape):
    """Each compiled tile configuration (pinned with sweep_config_select) of
    each pass length gives the oracle's sweeps on a ragged grid, and on one
    whose x extent is a whole number of 32-column tiles (the last column's
    right neighbour is the Dirichlet halo, read from the staged plane by the
    one-sweep tiles)."""
    u, f, h = rand_problem(*shape, seed=41)
    n = 8
    if dtype == S.F64:
        ref = oracle.jacobi(u, f, h, n)
        tol = FP64_TOL
        u_in, f_in = u, f
    elif dtype == S.F32:
        u_in, f_in = u.astype(np.float32).astype(np.float64), f.astype(np.float32).astype(np.float64)
        a = u.astype(np.float32)
        for _ in range(n):
            a = oracle.jacobi_sweep_f32(a, f.astype(np.float32), h)
        ref, tol = a.astype(np.float64), FP32_TOL
    else:
        u_in = oracle.from_bf16(oracle.to_bf16(u.astype(np.float32))).astype(np.float64)
        f_in = oracle.from_bf16(oracle.to_bf16(f.astype(np.float32))).astype(np.float64)
        ref, tol = oracle.jacobi(u_in, f_in, h, n), None
    c = S.Context(0)
    for T in range(1, 9):
        count = S.stencil_sweep_config_count(dtype, flags, with_work, T)
        for idx in range(count):
            S.stencil_sweep_config_select(c, dtype, flags, with_work, T, idx)
            uf, ff = S.Field.from_numpy(u_in, dtype), S.Field.from_numpy(f_in, dtype)
            w = S.Field(uf.nx, uf.ny, uf.nz) if with_work else None
            S.stencil_jacobi_sweep(c, uf, uf.like(), ff, w, h, n, T, flags)
            S.stencil_ctx_status(c)
            got = uf.to_numpy()
            t = tol if tol is not None else (-(-n // T)) * 2.0 ** -8
            assert rel_err(got, ref) <= t, (T, idx)
            assert halo_equal(got, u_in)
    c.close()


def test_autotune_then_parity():
    u, f, h = rand_problem(90, 61, 33, seed=42)
    c = S.Context(0)
    uf, ff = S.Field.from_numpy(u), S.Field.from_numpy(f)
    t, w = uf.like(), S.Field(uf.nx, uf.ny, uf.nz)
    rep = S.stencil_autotune_sweep(c, uf, t, ff, w, h)
    assert "chosen" in rep and "ms/sweep" in rep
    assert np.array_equal(uf.to_numpy(), u)  # the tuner does not change u
    S.stencil_jacobi_sweep(c, uf, t, ff, w, h, 12, 0, 0)
    S.stencil_ctx_status(c)
    assert rel_err(uf.to_numpy(), oracle.jacobi(u, f, h, 12)) <= FP64_TOL
    c.close()
