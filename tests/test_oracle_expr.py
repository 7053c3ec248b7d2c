"""Pins of the oracle's general stencil.apply (oracle/expr.py).

The evaluator is checked against what does not depend on it: closed forms
on integer-valued fields (where every binary64 operation is exact), the
linear apply oracle (a linear body written as an expression gives the same
binary64 operations in the same order), and the advection oracle (the
Piacsek-Williams tendencies written as expressions, with the vertical
factors as fields, give its values bit for bit).  A planted mistake in the
parser (a wrong precedence, a dropped sign, a shifted offset) fails one of
these."""
import numpy as np
import pytest

import oracle
from oracle import expr as E
from paper_2310_01882_b300 import inputs


def _int_field(nx, ny, nz):
    k, j, i = np.meshgrid(np.arange(nz + 2), np.arange(ny + 2), np.arange(nx + 2), indexing="ij")
    return (i * i + 2 * j - 3 * k).astype(np.float64), (i, j, k)


def test_closed_forms_on_an_integer_field():
    u, (i, j, k) = _int_field(9, 7, 6)
    inner = (slice(1, -1),) * 3
    d2x = E.apply_expr([u], "a0(1,0,0) - 2*a0(0,0,0) + a0(-1,0,0)")
    assert np.all(d2x[inner] == 2.0)
    dy = E.apply_expr([u], "(a0(0,1,0) - a0(0,-1,0)) / 2")
    assert np.all(dy[inner] == 2.0)
    dz = E.apply_expr([u], "a0(0,0,1) - a0(0,0,-1)")
    assert np.all(dz[inner] == -6.0)
    neg = E.apply_expr([u], "-a0(0,0,0) / 4")
    assert np.array_equal(neg[inner], -u[inner] / 4)
    prec = E.apply_expr([u], "1 + 2 * 3 - 8 / 4 / 2")  # precedence and left association
    assert np.all(prec[inner] == 6.0)
    two = E.apply_expr([u, 2 * u], "a1(0,0,0) - a0(0,0,0) * 2")
    assert np.all(two[inner] == 0.0)


def test_bounds_follow_the_radius_and_the_rest_is_untouched():
    u, _ = _int_field(8, 8, 8)
    out0 = np.full(u.shape, -7.0)
    got = E.apply_expr([u], "a0(2,0,0) - a0(-2,0,0)", out=out0)
    assert np.all(got[2:-2, 2:-2, 2:-2] == 8.0 * np.arange(2, 8)[None, None, :])
    mask = np.ones(u.shape, bool)
    mask[2:-2, 2:-2, 2:-2] = False
    assert np.all(got[mask] == -7.0)


@pytest.mark.parametrize("axis,r", [(0, 3), (1, 2), (2, 3), (2, 1)])
def test_the_largest_offset_on_any_axis_sets_the_bounds(axis, r):
    u, (i, _, _) = _int_field(9, 8, 10)
    d = [0, 0, 0]
    d[axis] = r
    expr = f"a0({d[0]},{d[1]},{d[2]}) - a0({-d[0]},{-d[1]},{-d[2]}) + a0(1,-1,1)*0"
    got = E.apply_expr([u], expr, out=np.full(u.shape, -7.0))
    inner = (slice(r, -r),) * 3
    # u = i^2 + 2j - 3k: the central difference over 2r cells
    want = 4 * r * i[inner] if axis == 0 else np.full(got[inner].shape, 2 * r * (2, -3)[axis - 1])
    assert np.array_equal(got[inner], want)
    mask = np.ones(u.shape, bool)
    mask[inner] = False
    assert np.all(got[mask] == -7.0)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_linear_body_equals_the_linear_apply_oracle(seed):
    rng = np.random.default_rng(seed)
    u = rng.standard_normal((12, 11, 13))
    offs = [tuple(int(v) for v in rng.integers(-2, 3, 3)) for _ in range(9)]
    coef = rng.standard_normal(9)
    expr = " + ".join(f"{float(c)!r}*a0({dx},{dy},{dz})" for c, (dx, dy, dz) in zip(coef, offs))
    out0 = rng.standard_normal(u.shape)
    assert np.array_equal(E.apply_expr([u], expr, out=out0), oracle.apply_linear(u, offs, coef, out=out0))


# The Piacsek-Williams tendencies (the advection oracle's formulas, its
# order of operations) over u, v, w = a0, a1, a2 and the vertical factors
# tzc1, tzc2 as fields a3, a4.
ADVECT_EXPR = {
    "su": "0.25*(a0(-1,0,0)*(a0(0,0,0)+a0(-1,0,0)) - a0(1,0,0)*(a0(0,0,0)+a0(1,0,0)))"
          " + 0.25*(a0(0,-1,0)*(a1(0,-1,0)+a1(1,-1,0)) - a0(0,1,0)*(a1(0,0,0)+a1(1,0,0)))"
          " + (a3(0,0,0)*a0(0,0,-1)*(a2(0,0,-1)+a2(1,0,-1)) - a4(0,0,0)*a0(0,0,1)*(a2(0,0,0)+a2(1,0,0)))",
    "sv": "0.25*(a1(-1,0,0)*(a0(-1,0,0)+a0(-1,1,0)) - a1(1,0,0)*(a0(0,0,0)+a0(0,1,0)))"
          " + 0.25*(a1(0,-1,0)*(a1(0,0,0)+a1(0,-1,0)) - a1(0,1,0)*(a1(0,0,0)+a1(0,1,0)))"
          " + (a3(0,0,0)*a1(0,0,-1)*(a2(0,0,-1)+a2(0,1,-1)) - a4(0,0,0)*a1(0,0,1)*(a2(0,0,0)+a2(0,1,0)))",
    "sw": "0.25*(a2(-1,0,0)*(a0(-1,0,0)+a0(-1,0,1)) - a2(1,0,0)*(a0(0,0,0)+a0(0,0,1)))"
          " + 0.25*(a2(0,-1,0)*(a1(0,-1,0)+a1(0,-1,1)) - a2(0,1,0)*(a1(0,0,0)+a1(0,0,1)))"
          " + (a3(0,0,0)*a2(0,0,-1)*(a2(0,0,0)+a2(0,0,-1)) - a4(0,0,0)*a2(0,0,1)*(a2(0,0,0)+a2(0,0,1)))",
}


def advect_inputs(nx, ny, nz, seeds=(4, 5, 6)):
    u, v, w = inputs.winds(nx, ny, nz, seeds=seeds)
    t1, t2 = inputs.tzc(nz, 7), inputs.tzc(nz, 8)
    f1, f2 = np.zeros_like(u), np.zeros_like(u)
    f1[1:-1] = t1[:, None, None]
    f2[1:-1] = t2[:, None, None]
    return (u, v, w, f1, f2), (t1, t2)


def test_advection_written_as_expressions_equals_the_advection_oracle():
    fields, (t1, t2) = advect_inputs(11, 9, 7)
    ref = oracle.advect_uvw(*fields[:3], t1, t2, 0.25, 0.25)
    inner = (slice(1, -1),) * 3
    for name, r in zip(("su", "sv", "sw"), ref):
        got = E.apply_expr(list(fields), ADVECT_EXPR[name])
        assert np.array_equal(got[inner], r[inner]), name


@pytest.mark.parametrize("bad", ["a0(4,0,0)", "a1(0,0,0)", "1 +", "a0(0,0)", "b0(0,0,0)", "((1)", "1e999", "2 3"])
def test_malformed_expressions_raise(bad):
    with pytest.raises(ValueError):
        E.apply_expr([np.zeros((5, 5, 5))], bad)
