"""Pins of the general linear stencil apply oracle: a single unit term is an
exact shift (catches a swapped axis or sign), the four-neighbour average
written as a linear stencil with coefficients 1/4 is bitwise the dedicated
average (scaling by 1/4 commutes with rounding), the 7-point Jacobi
average with f = 0 agrees to rounding, and a dense matrix built from the
offsets reproduces the apply."""
import itertools

import numpy as np
import pytest

import oracle


def field(shape, seed):
    nx, ny, nz = shape
    return np.random.default_rng(seed).standard_normal((nz + 2, ny + 2, nx + 2))


@pytest.mark.parametrize("d", list(itertools.product((-1, 0, 1), repeat=3)))
def test_unit_term_is_a_shift(d):
    u = field((5, 4, 3), 1)
    got = oracle.apply_linear(u, [d], [1.0])
    dx, dy, dz = d
    ref = u[1 + dz:u.shape[0] - 1 + dz, 1 + dy:u.shape[1] - 1 + dy, 1 + dx:u.shape[2] - 1 + dx]
    assert np.array_equal(got[1:-1, 1:-1, 1:-1], ref)


def test_four_neighbour_average_bitwise():
    u = field((13, 9, 2), 2)
    got = oracle.apply_linear(u, [(-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0)], [0.25] * 4)
    ref = oracle.average2d(u, 1)
    assert np.array_equal(got[1:-1, 1:-1, 1:-1], ref[1:-1, 1:-1, 1:-1])


def test_seven_point_average_matches_jacobi():
    u = field((7, 6, 5), 3)
    nb = [(-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]
    got = oracle.apply_linear(u, nb, [1.0 / 6.0] * 6)
    ref = oracle.jacobi_sweep(u, np.zeros_like(u), 0.1)
    assert np.max(np.abs(got[1:-1, 1:-1, 1:-1] - ref[1:-1, 1:-1, 1:-1])) <= 1e-15 * np.max(np.abs(u))


def test_dense_matrix():
    rng = np.random.default_rng(4)
    u = field((3, 4, 2), 5)
    offs = [tuple(int(v) for v in rng.integers(-1, 2, 3)) for _ in range(9)]
    coef = rng.standard_normal(9)
    got = oracle.apply_linear(u, offs, coef)
    nz, ny, nx = (s - 2 for s in u.shape)
    flat = u.reshape(-1)
    M = np.zeros((nx * ny * nz, flat.size))
    n = 0
    for k in range(1, nz + 1):
        for j in range(1, ny + 1):
            for i in range(1, nx + 1):
                for (dx, dy, dz), c in zip(offs, coef):
                    M[n, np.ravel_multi_index((k + dz, j + dy, i + dx), u.shape)] += c
                n += 1
    ref = (M @ flat).reshape(nz, ny, nx)
    assert np.max(np.abs(got[1:-1, 1:-1, 1:-1] - ref)) <= 1e-13


@pytest.mark.parametrize("d", [(2, 0, 0), (0, -2, 1), (-3, 1, 2), (1, 3, -3)])
def test_wide_unit_term_is_a_shift_on_the_shrunken_bounds(d):
    """Offsets beyond the one-cell halo: the output covers indices r .. n+1-r
    (r = max |d|), where every read lies in the field; nothing else is
    written."""
    u = field((9, 8, 7), 6)
    sentinel = np.full(u.shape, 7.5)
    got = oracle.apply_linear(u, [d], [1.0], out=sentinel)
    r = max(abs(v) for v in d)
    dx, dy, dz = d
    nz, ny, nx = (s - 2 for s in u.shape)
    core = (slice(r, nz + 2 - r), slice(r, ny + 2 - r), slice(r, nx + 2 - r))
    ref = u[r + dz:nz + 2 - r + dz, r + dy:ny + 2 - r + dy, r + dx:nx + 2 - r + dx]
    assert np.array_equal(got[core], ref)
    mask = np.ones(u.shape, dtype=bool)
    mask[core] = False
    assert np.all(got[mask] == 7.5)


def test_fourth_order_laplacian_exact_on_quintics():
    """The 13-point fourth-order Laplacian ((-1, 16, -30, 16, -1)/12 along
    each axis, unit spacing) is exact for polynomials of degree <= 5 in each
    variable: u = i^4 + 2 j^5 - k^3 gives 12 i^2 + 40 j^3 - 6 k on the
    points two cells inside."""
    nx, ny, nz = 10, 9, 8
    k, j, i = np.meshgrid(np.arange(nz + 2), np.arange(ny + 2), np.arange(nx + 2), indexing="ij")
    u = (i.astype(float) ** 4 + 2.0 * j.astype(float) ** 5 - k.astype(float) ** 3)
    w = [-1.0 / 12, 16.0 / 12, -30.0 / 12, 16.0 / 12, -1.0 / 12]
    offs, coef = [], []
    for axis in range(3):
        for s, c in zip(range(-2, 3), w):
            d = [0, 0, 0]
            d[axis] = s
            offs.append(tuple(d))
            coef.append(c)
    got = oracle.apply_linear(u, offs, coef)
    exact = 12.0 * i ** 2 + 40.0 * j ** 3 - 6.0 * k
    core = (slice(2, nz), slice(2, ny), slice(2, nx))
    assert np.max(np.abs(got[core] - exact[core])) <= 1e-9 * np.max(np.abs(u))


def test_dense_matrix_radius_two():
    rng = np.random.default_rng(8)
    u = field((6, 5, 5), 9)
    offs = [tuple(int(v) for v in rng.integers(-2, 3, 3)) for _ in range(11)] + [(2, 2, 2)]
    coef = rng.standard_normal(12)
    got = oracle.apply_linear(u, offs, coef)
    nz, ny, nx = (s - 2 for s in u.shape)
    flat = u.reshape(-1)
    rows, ref = [], []
    for k in range(2, nz):
        for j in range(2, ny):
            for i in range(2, nx):
                row = np.zeros(flat.size)
                for (dx, dy, dz), c in zip(offs, coef):
                    row[np.ravel_multi_index((k + dz, j + dy, i + dx), u.shape)] += c
                rows.append(row)
                ref.append(got[k, j, i])
    assert np.max(np.abs(np.array(rows) @ flat - np.array(ref))) <= 1e-13
