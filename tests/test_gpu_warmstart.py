"""The time-to-residual harness on the GPU: the plain FP64 baseline solver
(its shape tuned for the way it runs) and the batched mixed solve both bring
seeded problems to the FP64 relative residual 1e-8, checked by the library's
FP64 residual and, on the smallest problem, by the oracle's."""
import numpy as np
import pytest

import oracle
from paper_2310_01882_b300 import inputs
from paper_2310_01882_b300 import stencil as S
from paper_2310_01882_b300 import warmstart

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def solver():
    return warmstart.Solver(20, streams=2)


def test_baseline_solver_reaches_tolerance(solver):
    n = solver.n
    fs = warmstart.make_fields(n, [500, 501, 502])
    us = [S.Field(n, n, n) for _ in fs]
    info = solver.solve(us, fs, chunk=100)
    assert all(rel <= warmstart.RTOL for _, rel in info)
    assert all(sw % 100 == 0 and sw > 0 for sw, _ in info)
    # the oracle's FP64 residual of the first returned u
    u = us[0].to_numpy()
    f = inputs.grf(n, seed=500)
    rn, fn = oracle.residual(u, f, solver.h)
    assert rn / fn <= warmstart.RTOL * (1 + 1e-9)
    # the tuned choices are compiled configurations
    for (rb, k), (T, idx) in solver.choice.items():
        assert T in (1, 2) and idx >= 0


@pytest.mark.parametrize("kind", ["fp64", "f32", "bf16", "fp64rb", "f32rb"])
def test_solve_together_every_kind(solver, kind):
    n = solver.n
    fs = warmstart.make_fields(n, [600, 601])
    dt, sweeps, worst, ok = warmstart.solve_together(solver, fs, [None, None], kind, chunk=100,
                                                     sweeps_per_cycle=100)
    assert ok and worst <= warmstart.RTOL
    assert len(sweeps) == 2 and min(sweeps) > 0


def test_training_checkpoint_resumes_exactly(tmp_path):
    """Three epochs in one go, and a run stopped after one epoch then
    resumed from its checkpoint (in a fresh net) for the other two, give the
    same parameters and loss history bit for bit."""
    n = 16
    fs = warmstart.make_fields(n, [700 + i for i in range(6)])
    us = [S.Field.from_numpy(0.01 * inputs.grf(n, seed=800 + i)) for i in range(6)]
    ref = S.WsNet(2, [16, 32], n, seed=5)
    h_ref = warmstart.train(ref, fs, us, 3, 2, 1e-3, seed=3)
    a = S.WsNet(2, [16, 32], n, seed=5)
    warmstart.train(a, fs, us, 3, 2, 1e-3, seed=3, ckpt_dir=str(tmp_path), stop_after=1)
    b = S.WsNet(2, [16, 32], n, seed=77)
    h = warmstart.train(b, fs, us, 3, 2, 1e-3, seed=3, ckpt_dir=str(tmp_path))
    assert np.array_equal(b.get_params(), ref.get_params())
    assert h == h_ref
    for net in (ref, a, b):
        net.close()
