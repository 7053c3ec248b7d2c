"""GPU parity of stencil_average2d (the paper's Listing 1, four-neighbour
average per z plane): bitwise equal to the oracle, the boundary kept."""
import numpy as np
import pytest

import oracle
from paper_2310_01882_b300 import stencil as S
from tests.gpu_util import ctx

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape", [(1, 1, 1), (130, 67, 1), (64, 48, 3), (1025, 3, 1), (8192, 8192, 1)])
@pytest.mark.parametrize("nsweeps", [1, 2, 7])
def test_bitwise(shape, nsweeps):
    import torch
    if shape[0] == 8192 and nsweeps != 2:
        pytest.skip("one sweep count at full size")
    nx, ny, nz = shape
    rng = np.random.default_rng(nx + ny + nz + nsweeps)
    u0 = rng.standard_normal((nz + 2, ny + 2, nx + 2))
    u = S.Field.from_numpy(u0)
    S.stencil_average2d(ctx(), u, u.like(), nsweeps)
    torch.cuda.synchronize()
    got = u.to_numpy()
    ref = oracle.average2d(u0, nsweeps)
    assert np.array_equal(got, ref)


def test_arguments():
    u = S.Field(8, 8, 1)
    with pytest.raises(S.StencilError):
        S.stencil_average2d(ctx(), u, u, 1)
    with pytest.raises(S.StencilError):
        S.stencil_average2d(ctx(), u, S.Field(8, 8, 1, S.F32), 1)
