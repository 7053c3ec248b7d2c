"""GPU parity of stencil_batch_solve (mixed-precision refinement of a batch
of independent instances) against the refinement oracle."""
import numpy as np
import pytest

import oracle
from oracle import exact
from paper_2310_01882_b300 import inputs
from paper_2310_01882_b300 import stencil as S
from tests.gpu_util import ctx

pytestmark = pytest.mark.gpu

SIZES = [(8, 8, 8), (12, 9, 7), (20, 20, 20), (33, 17, 11), (16, 40, 9), (24, 24, 24)]


def make_batch(sizes, seed0):
    us, fs, hs, f_np = [], [], [], []
    for q, (nx, ny, nz) in enumerate(sizes):
        f = inputs.grf(nx, seed=seed0 + q, ny=ny, nz=nz)
        h = 1.0 / (max(nx, ny, nz) + 1)
        us.append(S.Field(nx, ny, nz))
        fs.append(S.Field.from_numpy(f))
        hs.append(h)
        f_np.append(f)
    return us, fs, hs, f_np


@pytest.mark.parametrize("smoother", ["jacobi", "redblack"])
@pytest.mark.parametrize("inner,name", [(S.F32, "f32"), (S.BF16, "bf16")])
def test_batch_matches_refinement_oracle(inner, name, smoother):
    import torch
    us, fs, hs, f_np = make_batch(SIZES, 100)
    res = S.stencil_batch_solve(ctx(), us, fs, hs, 1e-8, inner_dtype=inner, sweeps_per_cycle=40,
                                smoother={"jacobi": 0, "redblack": 1}[smoother])
    torch.cuda.synchronize()
    for q, (u, f, h, r) in enumerate(zip(us, f_np, hs, res)):
        ref = oracle.refine(np.zeros_like(f), f, h, 1e-8, inner=name, m=40, smoother=smoother)
        got = u.to_numpy()
        nr, nf = oracle.residual(got, f, h)
        assert r["status"] == 0 and ref["status"] == 0, (q, r, ref["status"])
        assert nr / nf <= 1e-8, (q, nr / nf)
        assert abs(r["rel_residual"] - nr / nf) <= 1e-12 * nr / nf + 1e-300
        assert abs(r["cycles"] - ref["cycles"]) <= 1, (q, r["cycles"], ref["cycles"])
        assert r["sweeps"] == r["cycles"] * 40
        ud = exact.solve(f, h)
        assert np.max(np.abs(got - ud)) <= 1e-5 * np.max(np.abs(ud))


def test_batch_budget_and_nonfinite():
    import torch
    us, fs, hs, f_np = make_batch([(10, 10, 10), (9, 7, 5), (6, 6, 6)], 200)
    bad = f_np[2].copy()
    bad[3, 3, 3] = np.inf
    fs[2] = S.Field.from_numpy(bad)
    res = S.stencil_batch_solve(ctx(), us, fs, hs, 1e-14, inner_dtype=S.F32, max_sweeps=80,
                                sweeps_per_cycle=40)
    torch.cuda.synchronize()
    assert res[0]["status"] == -7 and res[0]["sweeps"] == 80
    assert res[1]["status"] == -7 and res[1]["sweeps"] == 80
    assert res[2]["status"] == -6 and res[2]["sweeps"] == 0


def test_batch_u_start_and_halo_kept():
    """A nonzero start and a nonzero Dirichlet halo: the solution is the
    oracle's refinement from the same start; halo bits unchanged."""
    import torch
    rng = np.random.default_rng(5)
    nx, ny, nz = 14, 11, 9
    u0 = rng.random((nz + 2, ny + 2, nx + 2))
    f = rng.standard_normal((nz + 2, ny + 2, nx + 2))
    h = 1.0 / 15
    u = S.Field.from_numpy(u0)
    res = S.stencil_batch_solve(ctx(), [u], [S.Field.from_numpy(f)], [h], 1e-8, inner_dtype=S.F32,
                                sweeps_per_cycle=20)
    torch.cuda.synchronize()
    got = u.to_numpy()
    ref = oracle.refine(u0, f, h, 1e-8, inner="f32", m=20)
    assert res[0]["status"] == 0
    nr, nf = oracle.residual(got, f, h)
    assert nr / nf <= 1e-8
    m = np.ones(u0.shape, dtype=bool)
    m[1:-1, 1:-1, 1:-1] = False
    assert np.array_equal(got[m], u0[m])
    assert abs(res[0]["cycles"] - ref["cycles"]) <= 1
