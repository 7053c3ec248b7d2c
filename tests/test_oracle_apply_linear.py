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
