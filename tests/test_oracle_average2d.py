"""Pins of the 2D four-neighbour average oracle (the paper's Listing 1):
a sine mode decays by exactly (cos(p pi/(nx+1)) + cos(q pi/(ny+1)))/2 per
sweep, a dense matrix built from the neighbour relation reproduces a sweep,
z planes stay independent, and the boundary is kept."""
import numpy as np
import pytest

import oracle


@pytest.mark.parametrize("mode", [(1, 1), (3, 2), (7, 5)])
def test_sine_mode_decay(mode):
    nx, ny = 11, 8
    p, q = mode
    i = np.arange(nx + 2)[None, :]
    j = np.arange(ny + 2)[:, None]
    plane = np.sin(np.pi * p * i / (nx + 1)) * np.sin(np.pi * q * j / (ny + 1))
    plane[0], plane[-1], plane[:, 0], plane[:, -1] = 0, 0, 0, 0
    u = np.zeros((3, ny + 2, nx + 2))
    u[1] = plane
    mu = (np.cos(np.pi * p / (nx + 1)) + np.cos(np.pi * q / (ny + 1))) / 2.0
    for n in (1, 6):
        got = oracle.average2d(u, n)
        assert np.max(np.abs(got[1] - mu ** n * plane)) <= 1e-14


def test_dense_matrix_and_independent_planes():
    nx, ny, nz = 4, 3, 2
    rng = np.random.default_rng(1)
    u = rng.standard_normal((nz + 2, ny + 2, nx + 2))
    got = oracle.average2d(u, 1)
    for k in range(1, nz + 1):
        pts = [(j, i) for j in range(1, ny + 1) for i in range(1, nx + 1)]
        idx = {p: n for n, p in enumerate(pts)}
        M = np.zeros((len(pts), len(pts)))
        b = np.zeros(len(pts))
        for n, (j, i) in enumerate(pts):
            for dj, di in ((0, -1), (0, 1), (-1, 0), (1, 0)):
                qq = (j + dj, i + di)
                if qq in idx:
                    M[n, idx[qq]] = 0.25
                else:
                    b[n] += 0.25 * u[k][qq]
        x = np.array([u[k][p] for p in pts])
        ref = M @ x + b
        assert np.max(np.abs(np.array([got[k][p] for p in pts]) - ref)) <= 1e-14
    m = np.ones(u.shape, dtype=bool)
    m[1:-1, 1:-1, 1:-1] = False
    assert np.array_equal(got[m], u[m])
