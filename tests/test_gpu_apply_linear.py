"""GPU parity of stencil_apply_linear (a general linear stencil.apply):
bitwise equal to the oracle for random offset sets and coefficients, the
out halo untouched."""
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


def test_arguments():
    a = S.Field(8, 8, 8)
    with pytest.raises(S.StencilError):
        S.stencil_apply_linear(ctx(), a, a, [(0, 0, 0)], [1.0])          # in place
    with pytest.raises(S.StencilError):
        S.stencil_apply_linear(ctx(), a, a.like(), [(2, 0, 0)], [1.0])   # beyond the halo
    with pytest.raises(S.StencilError):
        S.stencil_apply_linear(ctx(), a, a.like(), [(0, 0, 0)] * 28, [1.0] * 28)
