"""stencil_residual_noalloc: the residual for callers that cannot allocate.

Some callers may not allocate device memory (they run inside a host program
that owns all device memory, or under a no-allocation policy) and so cannot
create a stencil_ctx.  The allocation-free entry point keeps its partial
sums in an array built into the library.  These tests call it through the C
ABI, twice in a row on different inputs (the shared array keeps the previous
call's contents), and compare with stencil_residual: r bitwise, the norms to
the tolerance the residual tests use (1e-13 relative).  The file is named to
be collected last; it also passes alone in a fresh process."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

NORM_TOL = 1e-13


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


def test_matches_context_residual_on_consecutive_calls():
    cases = [((130, 67, 45), 1), ((64, 64, 64), 2), ((7, 5, 3), 3)]
    for (nx, ny, nz), seed in cases:
        u, f = _fields(nx, ny, nz, seed)
        h = 1.0 / (max(nx, ny, nz) + 1)
        ref_n, ref_r = _with_ctx(u, f, h)
        got_n, got_r = _without_alloc(u, f, h)
        assert np.array_equal(got_r[1:-1, 1:-1, 1:-1], ref_r[1:-1, 1:-1, 1:-1])
        assert np.all(np.abs(got_n - ref_n) <= NORM_TOL * ref_n), (got_n, ref_n)


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
