"""Pins for the oracle's Piacsek-Williams advection (Section 4.1).

The expected values are closed forms derived by hand for fields that are
constant or linear in the grid indices (each of the nine direction terms is
exercised by one case, with distinct coefficients so that a wrong sign, a
swapped neighbour, a transposed axis or a swapped tzc1/tzc2 fails), plus the
telescoping of the self-advection term over a periodic line."""
import numpy as np
import pytest

import oracle
from paper_2310_01882_b300 import inputs

NX, NY, NZ = 9, 7, 6
TCX, TCY = 0.25, 0.3


def idx():
    k, j, i = np.meshgrid(np.arange(NZ + 2), np.arange(NY + 2), np.arange(NX + 2), indexing="ij")
    return i.astype(float), j.astype(float), k.astype(float)


def coeffs():
    rng = np.random.default_rng(8)
    return 0.5 + rng.random(NZ), 0.5 + rng.random(NZ)


def interior(a):
    return a[1:-1, 1:-1, 1:-1]


def run(u, v, w, t1, t2):
    return oracle.advect_uvw(u, v, w, t1, t2, TCX, TCY)


def test_constant_fields_zero_tendency():
    t = coeffs()[0]
    c = np.full((NZ + 2, NY + 2, NX + 2), 3.7)
    su, sv, sw = run(c, c, c, t, t)
    for s in (su, sv, sw):
        assert np.all(interior(s) == 0.0)
    # arbitrary tzc: u, v constant and w = 0 still give zero
    t1, t2 = coeffs()
    z = np.zeros_like(c)
    su, sv, sw = run(c, c, z, t1, t2)
    assert np.all(interior(su) == 0.0) and np.all(interior(sv) == 0.0) and np.all(interior(sw) == 0.0)
    # constant w and distinct tzc: sw = 2 c^2 (tzc1 - tzc2) per level
    su, sv, sw = run(z, z, c, t1, t2)
    expect = 2 * 3.7 ** 2 * (t1 - t2)
    np.testing.assert_allclose(interior(sw), np.broadcast_to(expect[:, None, None], (NZ, NY, NX)), rtol=1e-14)


def test_self_terms_linear():
    i, j, k = idx()
    a = 0.5
    t1, t2 = coeffs()
    z = np.zeros_like(i)
    su, _, _ = run(a * i, z, z, t1, t2)
    np.testing.assert_array_equal(interior(su), interior(-6 * a * a * i * TCX))
    _, sv, _ = run(z, a * j, z, t1, t2)
    np.testing.assert_array_equal(interior(sv), interior(-6 * a * a * j * TCY))
    _, _, sw = run(z, z, a * k, t1, t2)
    T1 = t1[:, None, None]
    T2 = t2[:, None, None]
    kk = interior(k)
    expect = a * a * (T1 * (2 * kk * kk - 3 * kk + 1) - T2 * (2 * kk * kk + 3 * kk + 1))
    np.testing.assert_allclose(interior(sw), expect, rtol=1e-13)


@pytest.mark.parametrize("b,c,d", [(1.5, 0.25, 0.125), (-0.75, 0.5, -0.25)])
def test_cross_terms_linear(b, c, d):
    i, j, k = idx()
    a = 0.5
    t1, t2 = coeffs()
    T1 = t1[:, None, None]
    T2 = t2[:, None, None]
    z = np.zeros_like(i)
    I, J, K = interior(i), interior(j), interior(k)
    # su, y term: u = a j, v = b + c i + d j
    su, _, _ = run(a * j, b + c * i + d * j, z, t1, t2)
    C = 2 * b + c * (2 * I + 1)
    np.testing.assert_allclose(interior(su), TCY * (-2 * a * C - 2 * a * d * (3 * J - 1)), rtol=1e-13, atol=1e-13)
    # su, z term: u = a k, w = b + c i + d k
    su, _, _ = run(a * k, z, b + c * i + d * k, t1, t2)
    expect = a * (T1 * (K - 1) * (C + 2 * d * (K - 1)) - T2 * (K + 1) * (C + 2 * d * K))
    np.testing.assert_allclose(interior(su), expect, rtol=1e-13, atol=1e-13)
    # sv, x term: v = a i, u = b + c j + d i
    _, sv, _ = run(b + c * j + d * i, a * i, z, t1, t2)
    Cj = 2 * b + c * (2 * J + 1)
    np.testing.assert_allclose(interior(sv), TCX * (-2 * a * Cj - 2 * a * d * (3 * I - 1)), rtol=1e-13, atol=1e-13)
    # sv, z term: v = a k, w = b + c j + d k
    _, sv, _ = run(z, a * k, b + c * j + d * k, t1, t2)
    expect = a * (T1 * (K - 1) * (Cj + 2 * d * (K - 1)) - T2 * (K + 1) * (Cj + 2 * d * K))
    np.testing.assert_allclose(interior(sv), expect, rtol=1e-13, atol=1e-13)
    # sw, x term: w = a i, u = b + c k + d i   (plus the z self term 2 a^2 i^2 (tzc1 - tzc2))
    _, _, sw = run(b + c * k + d * i, z, a * i, t1, t2)
    Ck = 2 * b + c * (2 * K + 1)
    expect = TCX * (-2 * a * Ck - 2 * a * d * (3 * I - 1)) + 2 * a * a * I * I * (T1 - T2)
    np.testing.assert_allclose(interior(sw), expect, rtol=1e-13, atol=1e-13)
    # sw, y term: w = a j, v = b + c k + d j
    _, _, sw = run(z, b + c * k + d * j, a * j, t1, t2)
    expect = TCY * (-2 * a * Ck - 2 * a * d * (3 * J - 1)) + 2 * a * a * J * J * (T1 - T2)
    np.testing.assert_allclose(interior(sw), expect, rtol=1e-13, atol=1e-13)


def test_self_term_telescopes_on_periodic_line():
    """With v = w = 0 and u periodic in x, sum_i su over each x line is 0;
    likewise sum_j sv with u = w = 0 and v periodic in y."""
    rng = np.random.default_rng(9)
    t1, t2 = coeffs()
    u = inputs.fill_periodic_xy(rng.standard_normal((NZ + 2, NY + 2, NX + 2)))
    z = np.zeros_like(u)
    su, _, _ = run(u, z, z, t1, t2)
    assert np.max(np.abs(interior(su).sum(axis=2))) <= 1e-13 * np.max(np.abs(su))
    _, sv, _ = run(z, u, z, t1, t2)
    assert np.max(np.abs(interior(sv).sum(axis=1))) <= 1e-13 * np.max(np.abs(sv))


def test_self_terms_antisymmetric_under_reflection():
    """Reflecting a direction and negating the advected component maps each
    self-advection term to minus its value at the mirrored cell: with
    u'[i] = -u[N+1-i] along a periodic x line (v = w = 0), su'(i) =
    -su(N+1-i); likewise sv along a periodic y line, and sw along z with
    zero halo planes and tzc1 = tzc2 constant.  Exact in binary64 (the
    same products, negated)."""
    rng = np.random.default_rng(12)
    z = np.zeros((NZ + 2, NY + 2, NX + 2))
    t = np.full(NZ, 0.8)
    # x: periodic halo, random interior
    u = inputs.fill_periodic_xy(np.pad(rng.standard_normal((NZ, NY, NX)), 1))
    ur = -u[:, :, ::-1].copy()
    su, _, _ = run(u, z, z, t, t)
    sur, _, _ = run(ur, z, z, t, t)
    np.testing.assert_array_equal(interior(sur), -interior(su)[:, :, ::-1])
    # y
    v = inputs.fill_periodic_xy(np.pad(rng.standard_normal((NZ, NY, NX)), 1))
    vr = -v[:, ::-1, :].copy()
    _, sv, _ = run(z, v, z, t, t)
    _, svr, _ = run(z, vr, z, t, t)
    np.testing.assert_array_equal(interior(svr), -interior(sv)[:, ::-1, :])
    # z: zero halo planes stay zero under the reflection
    w = np.pad(rng.standard_normal((NZ, NY, NX)), 1)
    w[:, 0, :], w[:, -1, :], w[:, :, 0], w[:, :, -1] = 0, 0, 0, 0
    wr = -w[::-1, :, :].copy()
    _, _, sw = run(z, z, w, t, t)
    _, _, swr = run(z, z, wr, t, t)
    np.testing.assert_array_equal(interior(swr), -interior(sw)[::-1, :, :])


def test_operation_count_is_the_papers_63():
    """The oracle's formula has exactly the paper's 63 floating-point
    operations per cell (Section 4.1): counting + - * in the three
    tendencies' statements, with every field access AT(...) as one operand,
    gives 21 per component (6 for x, 6 for y, 7 for z, 2 to combine)."""
    import os
    import re
    src = open(os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle",
                            "oracle.c")).read()
    body = src[src.index("void oracle_advect_uvw"):]
    body = body[body.index("/* u component"):body.index("AT(sw, i, j, k) = tx + ty + tz;") + 40]
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    body = re.sub(r"AT\([^()]*\)", "X", body)
    parts = body.split("X = tx + ty + tz;")
    per = [len(re.findall(r"[+\-*]", p)) + 2 for p in parts[:3]]  # + the two adds that combine
    assert per == [21, 21, 21], per
    assert len(re.findall(r"[+\-*]", body)) == 63
