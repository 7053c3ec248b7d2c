"""stencil_residual_noalloc: the residual for callers that cannot allocate.

Some callers may not allocate device memory (they run inside a host program
that owns all device memory, or under a no-allocation policy) and so cannot
create a stencil_ctx.  The allocation-free entry point keeps its partial
sums in an array built into the library.  These tests call it through the C
ABI, twice in a row on different inputs (the shared array keeps the previous
call's contents), and compare with the CPU oracle (r bitwise: this entry
point evaluates the definition in its written order; the norms to 1e-12, a
different summation order) and with stencil_residual (the fixed-point
evaluation: r and the norms within both evaluations' rounding bound).  The
file is named to be collected last; it also passes alone in a fresh
process."""
import numpy as np
import pytest

import oracle

pytestmark = pytest.mark.gpu

NORM_TOL = 1e-13
ORACLE_NORM_TOL = 1e-12


def _fields(nx, ny, nz, seed):
    from paper_2310_01882_b300 import stencil as S
    rng = np.random.default_rng(seed)
    u = rng.random((nz + 2, ny + 2, nx + 2))
    f = rng.standard_normal((nz + 2, ny + 2, nx + 2))
    return S.Field.from_numpy(u), S.Field.from_numpy(f)


def _with_ctx(u, f, h):
    import torch
    from paper_2310_01882_b300 import stencil as S
    ctx = S.Context(0)
    norms = torch.zeros(2, dtype=torch.float64, device="cuda")
    r = S.Field(u.nx, u.ny, u.nz)
    S.stencil_residual(ctx, u, f, h, norms, r=r)
    torch.cuda.synchronize()
    ctx.close()
    return norms.cpu().numpy(), r.to_numpy()


def _without_alloc(u, f, h):
    import torch
    from paper_2310_01882_b300 import stencil as S
    norms = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    r = S.Field(u.nx, u.ny, u.nz)
    S.stencil_residual_noalloc(u, f, h, norms, r=r)
    torch.cuda.synchronize()
    return norms.cpu().numpy(), r.to_numpy()


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2310_01882_b300 import build
    build.build()


def _check(u, f, h):
    ref_n, ref_r = _with_ctx(u, f, h)
    got_n, got_r = _without_alloc(u, f, h)
    un, fn = u.to_numpy(), f.to_numpy()
    tol = 1e-14 * (12.0 * np.max(np.abs(un)) / (h * h) + np.max(np.abs(fn[1:-1, 1:-1, 1:-1])))
    assert np.max(np.abs(got_r[1:-1, 1:-1, 1:-1] - ref_r[1:-1, 1:-1, 1:-1])) <= tol
    assert abs(got_n[0] - ref_n[0]) <= np.sqrt(un[1:-1, 1:-1, 1:-1].size) * tol + NORM_TOL * ref_n[0]
    assert abs(got_n[1] - ref_n[1]) <= NORM_TOL * ref_n[1]
    on_r, on_f, o_r = oracle.residual(un, fn, h, want_r=True, nthreads=0)
    assert np.array_equal(got_r[1:-1, 1:-1, 1:-1], o_r[1:-1, 1:-1, 1:-1])
    assert abs(got_n[0] - on_r) <= ORACLE_NORM_TOL * on_r and abs(got_n[1] - on_f) <= ORACLE_NORM_TOL * on_f


def test_matches_context_residual_and_oracle_on_consecutive_calls():
    cases = [((130, 67, 45), 1), ((64, 64, 64), 2), ((7, 5, 3), 3)]
    for (nx, ny, nz), seed in cases:
        u, f = _fields(nx, ny, nz, seed)
        _check(u, f, 1.0 / (max(nx, ny, nz) + 1))


def test_at_the_limit_every_partial_sum_in_use():
    """ny * nz = 524288 rows: 8192 blocks, every pair of the built-in array."""
    u, f = _fields(4, 512, 1024, 7)
    _check(u, f, 1.0 / 1025)


def test_a_warm_call_allocates_nothing():
    """Device free memory is unchanged across a call (after a first call has
    loaded the library's kernels)."""
    import torch
    from paper_2310_01882_b300 import stencil as S
    u, f = _fields(70, 33, 21, 4)
    norms = torch.zeros(2, dtype=torch.float64, device="cuda")
    S.stencil_residual_noalloc(u, f, 0.01, norms)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    S.stencil_residual_noalloc(u, f, 0.01, norms)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0


def test_rejects_output_aliasing_an_input():
    import torch
    from paper_2310_01882_b300 import stencil as S
    u, f = _fields(9, 8, 7, 5)
    norms = torch.zeros(2, dtype=torch.float64, device="cuda")
    for r in (u, f):
        with pytest.raises(S.StencilError) as e:
            S.stencil_residual_noalloc(u, f, 0.1, norms, r=r)
        assert e.value.code == -1 and "aliases" in str(e.value)


def test_rejects_grid_beyond_scratch():
    import torch
    from paper_2310_01882_b300 import stencil as S
    u = S.Field(1, 1, 524289)   # ny * nz = 524289 rows, one beyond the limit
    f = S.Field(1, 1, 524289)
    norms = torch.zeros(2, dtype=torch.float64, device="cuda")
    with pytest.raises(S.StencilError) as e:
        S.stencil_residual_noalloc(u, f, 0.1, norms)
    assert e.value.code == -1 and "524288" in str(e.value)
    # at the limit it runs
    u = S.Field(1, 1, 524288)
    f = S.Field(1, 1, 524288)
    S.stencil_residual_noalloc(u, f, 0.1, norms)
    torch.cuda.synchronize()
