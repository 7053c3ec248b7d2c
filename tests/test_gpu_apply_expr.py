"""GPU parity of stencil_apply_expr, the general stencil.apply whose kernel
is generated from an expression and compiled at run time: bitwise equal to
the oracle's binary64 evaluation (oracle/expr.py) for linear and non-linear
bodies, several inputs, offsets up to three cells and ragged grids; the
Piacsek-Williams tendencies written as expressions equal the advection
oracle bit for bit; points outside the bounds are untouched; compiled
kernels are reused; malformed calls are rejected before any launch."""
import numpy as np
import pytest

import oracle
from oracle import expr as E
from paper_2310_01882_b300 import stencil as S
from tests.gpu_util import ctx
from tests.test_oracle_expr import ADVECT_EXPR, advect_inputs

pytestmark = pytest.mark.gpu

EXPRS = [
    ("0.25*(a0(-1,0,0) + a0(1,0,0) + a0(0,-1,0) + a0(0,1,0))", 1),
    ("a0(0,0,0)*a0(0,0,0) - a1(1,0,0)/(1 + a1(0,0,0)*a1(0,0,0))", 2),
    ("-(a0(0,0,1) - a0(0,0,-1)) * 0.5 + a2(3,0,0) - 3*a2(0,-3,2)", 3),
    ("(16*(a0(1,0,0) + a0(-1,0,0)) - (a0(2,0,0) + a0(-2,0,0)) - 30*a0(0,0,0)) / 12", 1),
    ("1.e2*a0(0,0,0) - .5E-1 + 7. / 3 * 0.1", 1),  # literals round-trip to the same binary64 values
    (" + ".join(f"a{q}({q % 3 - 1},{(q // 3) % 3 - 1},{q % 2})" for q in range(8)) + " * a7(0,0,-1)", 8),
]
SHAPES = [(1, 1, 1), (9, 8, 7), (67, 35, 19), (130, 17, 40)]


def run(c, fields, expr, out0):
    import torch
    ins = [S.Field.from_numpy(a) for a in fields]
    out = S.Field.from_numpy(out0)
    S.stencil_apply_expr(c, ins, out, expr)
    torch.cuda.synchronize()
    S.stencil_ctx_status(c)
    return out.to_numpy()


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("case", range(len(EXPRS)))
def test_bitwise_the_oracle(shape, case):
    expr, nin = EXPRS[case]
    nx, ny, nz = shape
    rng = np.random.default_rng(100 + case + nx)
    fields = [rng.standard_normal((nz + 2, ny + 2, nx + 2)) for _ in range(nin)]
    out0 = rng.standard_normal(fields[0].shape)
    got = run(ctx(), fields, expr, out0)
    assert np.array_equal(got, E.apply_expr(fields, expr, out=out0))


def test_advection_as_expressions_equals_the_advection_oracle():
    fields, (t1, t2) = advect_inputs(45, 37, 13)
    ref = oracle.advect_uvw(*fields[:3], t1, t2, 0.25, 0.25)
    inner = (slice(1, -1),) * 3
    for name, r in zip(("su", "sv", "sw"), ref):
        got = run(ctx(), list(fields), ADVECT_EXPR[name], np.zeros_like(r))
        assert np.array_equal(got[inner], r[inner]), name


def test_kernels_are_reused_and_results_repeat():
    rng = np.random.default_rng(7)
    u = rng.standard_normal((12, 11, 10))
    a, b = EXPRS[0][0], EXPRS[3][0]
    first = run(ctx(), [u], a, np.zeros_like(u))
    run(ctx(), [u], b, np.zeros_like(u))
    again = run(ctx(), [u], a, np.zeros_like(u))
    assert np.array_equal(first, again)


def test_rejected_calls():
    u, v = S.Field(8, 8, 8), S.Field(8, 8, 8)
    for expr in ("a0(4,0,0)", "a1(0,0,0)", "1 +"):
        with pytest.raises(S.StencilError) as e:
            S.stencil_apply_expr(ctx(), [u], v, expr)
        assert e.value.code == -1
    with pytest.raises(S.StencilError):
        S.stencil_apply_expr(ctx(), [u, v], v, "a0(0,0,0)")   # out aliases an input
    with pytest.raises(S.StencilError):
        S.stencil_apply_expr(ctx(), [u, S.Field(8, 8, 9)], v, "a0(0,0,0)")  # extents differ
