"""GPU parity of stencil_apply_linear (a general linear stencil.apply, offsets
up to three cells): with general coefficients (binary64 in the written
order) bitwise equal to the oracle, the rest of out untouched; with
integer-weight coefficients (the fixed-point path) exact -- bitwise equal to
the oracle on integer-valued inputs, where both are exact -- and within the
oracle's own rounding bound otherwise."""
import numpy as np
import pytest

import oracle
from paper_2310_01882_b300 import stencil as S
from tests.gpu_util import ctx

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape", [(1, 1, 1), (67, 35, 19), (130, 17, 7), (256, 256, 64)])
@pytest.mark.parametrize("npoints", [1, 7, 27])
def test_bitwise(shape, npoints):
    import torch
    nx, ny, nz = shape
    rng = np.random.default_rng(nx + npoints)
    u = rng.standard_normal((nz + 2, ny + 2, nx + 2))
    if npoints == 27:
        offs = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]
    else:
        offs = [tuple(int(v) for v in rng.integers(-1, 2, 3)) for _ in range(npoints)]
    coef = rng.standard_normal(npoints)
    out0 = rng.standard_normal(u.shape)
    a, b = S.Field.from_numpy(u), S.Field.from_numpy(out0)
    S.stencil_apply_linear(ctx(), a, b, offs, coef)
    torch.cuda.synchronize()
    got = b.to_numpy()
    ref = oracle.apply_linear(u, offs, coef, out=out0)
    assert np.array_equal(got, ref)


def run(u, offs, coef, out0):
    import torch
    a, b = S.Field.from_numpy(u), S.Field.from_numpy(out0)
    S.stencil_apply_linear(ctx(), a, b, offs, coef)
    torch.cuda.synchronize()
    S.stencil_ctx_status(ctx())
    return b.to_numpy()


def star(radius, weights):
    """Offsets and coefficients of a star stencil: weights[d] at distance d
    along each axis (weights[0] at the centre once)."""
    offs, coef = [(0, 0, 0)], [weights[0]]
    for axis in range(3):
        for d in range(1, radius + 1):
            for sgn in (-1, 1):
                o = [0, 0, 0]
                o[axis] = sgn * d
                offs.append(tuple(o))
                coef.append(weights[d])
    return offs, coef


@pytest.mark.parametrize("shape", [(9, 8, 7), (67, 35, 19), (130, 17, 9)])
@pytest.mark.parametrize("radius", [2, 3])
def test_wide_offsets_bitwise(shape, radius):
    """General coefficients, offsets up to `radius`: bitwise the oracle; out
    is written only on the points whose reads lie in the field."""
    nx, ny, nz = shape
    rng = np.random.default_rng(nx + radius)
    u = rng.standard_normal((nz + 2, ny + 2, nx + 2))
    offs = [tuple(int(v) for v in rng.integers(-radius, radius + 1, 3)) for _ in range(12)]
    offs.append((radius, -radius, radius))
    coef = rng.standard_normal(len(offs))
    out0 = rng.standard_normal(u.shape)
    assert np.array_equal(run(u, offs, coef, out0), oracle.apply_linear(u, offs, coef, out=out0))


INT_STENCILS = {
    "laplacian7": star(1, [-6.0, 1.0]),
    "laplacian13_4th": star(2, [-90.0, 16.0, -1.0]),       # 12 h^2 times the fourth-order Laplacian
    "star19_r3": star(3, [-25.0, 3.0, -2.0, 1.0]),
    # stars whose weights differ by axis and sign (the general star path) and
    # a symmetric one with a zero weight at one distance
    "star13_uneven": (star(2, [0.0] * 3)[0],
                      [float(v) for v in np.random.default_rng(1).integers(-40, 41, 13)]),
    "star19_uneven_r3": (star(3, [0.0] * 4)[0],
                         [float(v) for v in np.random.default_rng(2).integers(-40, 41, 19)]),
    "star13_sym_zero_d2": star(2, [4.0, -1.0, 0.0]),
    "average4": ([(-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0)], [0.25] * 4),
    "box27": ([(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)],
              [float(v) for v in np.random.default_rng(0).integers(-9, 10, 27)]),
    # off-axis offsets of radius 2, a repeated offset, a zero weight: the
    # fixed-point kernel that reads its terms at run time
    "random_r2": ([(1, -2, 0), (0, 0, 0), (-1, 1, 2), (2, 2, -1), (1, -2, 0), (0, -2, 1)],
                  [3.0, -8.0, 0.5, -1.25, 2.0, 0.0]),
}


@pytest.mark.parametrize("name", sorted(INT_STENCILS))
@pytest.mark.parametrize("shape", [(9, 8, 7), (67, 35, 19), (130, 17, 40)])
def test_integer_weights_exact_on_integer_inputs(name, shape):
    """Integer-valued inputs and integer (or dyadic) weights: every partial
    sum is exact in both evaluations, so the fixed-point path must equal the
    oracle bit for bit -- every offset, index and bound is checked."""
    nx, ny, nz = shape
    offs, coef = INT_STENCILS[name]
    rng = np.random.default_rng(sum(shape) + len(offs))
    u = rng.integers(-1000, 1001, (nz + 2, ny + 2, nx + 2)).astype(np.float64)
    out0 = rng.standard_normal(u.shape)
    assert np.array_equal(run(u, offs, coef, out0), oracle.apply_linear(u, offs, coef, out=out0))


@pytest.mark.parametrize("name", ["laplacian7", "laplacian13_4th", "star19_r3", "star13_uneven", "box27", "random_r2"])
@pytest.mark.parametrize("shape", [(1, 1, 1), (2, 3, 2), (3, 3, 3), (1, 40, 33), (37, 1, 5), (5, 6, 1)])
def test_integer_weights_tiny_and_thin_grids(name, shape):
    """Grids whose output bounds are empty, a single point or one cell
    thick at the stencil's radius: the fixed-point paths write exactly the
    oracle's points (bitwise on integer-valued inputs) and nothing else."""
    nx, ny, nz = shape
    offs, coef = INT_STENCILS[name]
    rng = np.random.default_rng(sum(shape) * 7 + len(offs))
    u = rng.integers(-1000, 1001, (nz + 2, ny + 2, nx + 2)).astype(np.float64)
    out0 = rng.standard_normal(u.shape)
    assert np.array_equal(run(u, offs, coef, out0), oracle.apply_linear(u, offs, coef, out=out0))


@pytest.mark.parametrize("name", sorted(INT_STENCILS))
def test_integer_weights_on_smooth_and_random_fields(name):
    """General binary64 inputs: the fixed-point sum is exact up to the
    input's conversion (2^-61 of sum |c| max|u|), the oracle's within
    npoints eps sum |c| max|u|; they agree to that bound (a smooth field,
    whose Laplacian cancels most digits, and a random one)."""
    offs, coef = INT_STENCILS[name]
    nx, ny, nz = 64, 48, 40
    k, j, i = np.meshgrid(np.arange(nz + 2), np.arange(ny + 2), np.arange(nx + 2), indexing="ij")
    smooth = np.sin(0.07 * i) * np.cos(0.05 * j) * np.sin(0.03 * k + 0.2) * 3.0
    rnd = np.random.default_rng(5).standard_normal(smooth.shape)
    for u in (smooth, rnd):
        out0 = np.zeros_like(u)
        got = run(u, offs, coef, out0)
        ref = oracle.apply_linear(u, offs, coef, out=out0)
        bound = 2 * len(offs) * np.finfo(float).eps * np.sum(np.abs(coef)) * np.max(np.abs(u))
        assert np.max(np.abs(got - ref)) <= bound, name


@pytest.mark.parametrize("name", ["laplacian13_4th", "box27"])
def test_scale_follows_each_input(name):
    """The fixed-point apply takes its scale from the magnitude of what its
    pass reads.  A context reuses the previous call's magnitude as the guess
    and repeats the pass when the guess gives another scale.  On one
    context, fields of very different magnitudes in turn (1e-150, 1e+150,
    1, 1 again, 1e-150 again) each stay within the oracle's rounding bound
    and equal bit for bit a fresh context's first call on the same input."""
    import torch
    offs, coef = INT_STENCILS[name]
    nx, ny, nz = 40, 33, 21
    base = np.random.default_rng(12).standard_normal((nz + 2, ny + 2, nx + 2))
    shared = S.Context(0)

    def go(c, u):
        a, b = S.Field.from_numpy(u), S.Field.from_numpy(np.zeros_like(u))
        S.stencil_apply_linear(c, a, b, offs, coef)
        torch.cuda.synchronize()
        S.stencil_ctx_status(c)
        return b.to_numpy()

    for scale in (1e-150, 1e150, 1.0, 1.0, 1e-150):
        u = scale * base
        got = go(shared, u)
        ref = oracle.apply_linear(u, offs, coef, out=np.zeros_like(u))
        bound = 2 * len(offs) * np.finfo(float).eps * np.sum(np.abs(coef)) * np.max(np.abs(u))
        assert np.max(np.abs(got - ref)) <= bound, scale
        fresh = S.Context(0)
        assert np.array_equal(got, go(fresh, u)), scale
        fresh.close()
    shared.close()


def test_full_size_benchmark_launch():
    """The benchmark's linear applies at full size: the 7-point and the
    fourth-order 13-point Laplacians on the 512^3 U[0,1) field (seed 3), two
    calls each on one context as bench.py times them (the first takes its
    scale from a range pass, the second from the first's magnitude): both
    within the oracle's rounding bound and equal bit for bit."""
    import torch
    from paper_2310_01882_b300 import inputs
    n = 512
    u = inputs.uniform(n, n, n, seed=3)
    c = S.Context(0)
    a = S.Field.from_numpy(u)
    b = a.like()
    for name in ("laplacian7", "laplacian13_4th"):
        offs, coef = INT_STENCILS[name]
        outs = []
        for _ in range(2):
            S.stencil_apply_linear(c, a, b, offs, coef)
            torch.cuda.synchronize()
            S.stencil_ctx_status(c)
            outs.append(b.to_numpy())
        ref = oracle.apply_linear(u, offs, coef, out=outs[0].copy())
        bound = 2 * len(offs) * np.finfo(float).eps * np.sum(np.abs(coef)) * np.max(np.abs(u))
        assert np.max(np.abs(outs[0] - ref)) <= bound, name
        assert np.array_equal(outs[0], outs[1]), name
    c.close()


def test_nonfinite_then_finite():
    """A NaN (or an infinity) in the input of the fixed-point apply: every
    output point is NaN and the context reports STENCIL_ERR_NONFINITE; the
    next call on the same context, with finite input, is right again."""
    import torch
    offs, coef = INT_STENCILS["laplacian13_4th"]
    rng = np.random.default_rng(83)
    u = rng.integers(-1000, 1001, (14, 13, 17)).astype(np.float64)
    c = S.Context(0)
    for bad in (np.nan, np.inf):
        ub = u.copy()
        ub[6, 6, 6] = bad
        a, b = S.Field.from_numpy(ub), S.Field.from_numpy(np.zeros_like(u))
        S.stencil_apply_linear(c, a, b, offs, coef)
        torch.cuda.synchronize()
        got = b.to_numpy()
        assert np.isnan(got[2:-2, 2:-2, 2:-2]).all()
        with pytest.raises(S.StencilError) as e:
            S.stencil_ctx_status(c)
        assert e.value.code == -6
        S.stencil_ctx_status(c)  # cleared
        a, b = S.Field.from_numpy(u), S.Field.from_numpy(np.zeros_like(u))
        S.stencil_apply_linear(c, a, b, offs, coef)
        torch.cuda.synchronize()
        S.stencil_ctx_status(c)
        assert np.array_equal(b.to_numpy(), oracle.apply_linear(u, offs, coef, out=np.zeros_like(u)))
    c.close()


def test_arguments():
    a = S.Field(8, 8, 8)
    with pytest.raises(S.StencilError):
        S.stencil_apply_linear(ctx(), a, a, [(0, 0, 0)], [1.0])          # in place
    with pytest.raises(S.StencilError):
        S.stencil_apply_linear(ctx(), a, a.like(), [(4, 0, 0)], [1.0])   # beyond three cells
    with pytest.raises(S.StencilError):
        S.stencil_apply_linear(ctx(), a, a.like(), [(0, 0, 0)] * 65, [1.0] * 65)
