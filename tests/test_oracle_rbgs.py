"""Pins of the red-black Gauss-Seidel oracle against what the mathematics
fixes (no GPU):
  * the block splitting, built densely from the neighbour relation on small
    grids (red unknowns first, then black), reproduces the in-place sweeps;
  * for f = 0 and a zero halo, a Jacobi eigenmode s with eigenvalue mu,
    taken with its black values scaled by mu, is an eigenvector of the
    red-black sweep with eigenvalue mu^2 (the classical relation for a
    consistently ordered matrix): it decays by exactly mu^2 per sweep;
  * the exact discrete solution is a fixed point, and the sweeps converge
    to the DST-I solution;
  * the FP32 and bf16 storage variants follow the FP64 one to their
    precision.
"""
import numpy as np
import pytest

import oracle
from oracle import exact


def coords(nx, ny, nz):
    k, j, i = np.meshgrid(np.arange(nz + 2), np.arange(ny + 2), np.arange(nx + 2), indexing="ij")
    return i, j, k


def dense_rb(u, f, h, nsweeps):
    """The red-black sweep as matrix algebra on the interior unknowns."""
    nz, ny, nx = (s - 2 for s in u.shape)
    idx = -np.ones(u.shape, dtype=np.int64)
    pts = [(k, j, i) for k in range(1, nz + 1) for j in range(1, ny + 1) for i in range(1, nx + 1)]
    for n, p in enumerate(pts):
        idx[p] = n
    N = len(pts)
    adj = np.zeros((N, N))
    bc = np.zeros(N)
    for n, (k, j, i) in enumerate(pts):
        for dk, dj, di in ((0, 0, -1), (0, 0, 1), (0, -1, 0), (0, 1, 0), (-1, 0, 0), (1, 0, 0)):
            q = (k + dk, j + dj, i + di)
            if idx[q] >= 0:
                adj[n, idx[q]] = 1.0
            else:
                bc[n] += u[q]
    color = np.array([(i + j + k) & 1 for (k, j, i) in pts])
    R, B = np.where(color == 0)[0], np.where(color == 1)[0]
    g = bc + h * h * np.array([f[p] for p in pts])
    x = np.array([u[p] for p in pts])
    for _ in range(nsweeps):
        x[R] = (adj[np.ix_(R, B)] @ x[B] + g[R]) / 6.0
        x[B] = (adj[np.ix_(B, R)] @ x[R] + g[B]) / 6.0
    out = u.copy()
    for n, p in enumerate(pts):
        out[p] = x[n]
    return out


@pytest.mark.parametrize("shape", [(4, 4, 4), (3, 5, 2), (5, 2, 3)])
def test_dense_splitting(shape):
    nx, ny, nz = shape
    rng = np.random.default_rng(nx * 100 + ny * 10 + nz)
    u = rng.standard_normal((nz + 2, ny + 2, nx + 2))  # nonzero halo: Dirichlet data
    f = rng.standard_normal(u.shape)
    h = 0.37
    for n in (1, 3):
        ref = dense_rb(u, f, h, n)
        got = oracle.rbgs(u, f, h, n)
        assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))
        assert np.array_equal(got[0], u[0]) and np.array_equal(got[:, :, -1], u[:, :, -1])


@pytest.mark.parametrize("mode", [(1, 1, 1), (2, 1, 3), (5, 4, 2)])
def test_eigenmode_decays_by_mu_squared(mode):
    nx, ny, nz = 9, 7, 6
    p, q, r = mode
    i, j, k = coords(nx, ny, nz)
    s = (np.sin(np.pi * p * i / (nx + 1)) * np.sin(np.pi * q * j / (ny + 1))
         * np.sin(np.pi * r * k / (nz + 1)))
    mu = (np.cos(np.pi * p / (nx + 1)) + np.cos(np.pi * q / (ny + 1)) + np.cos(np.pi * r / (nz + 1))) / 3.0
    y0 = np.where(((i + j + k) & 1) == 1, mu * s, s)
    y0[0], y0[-1], y0[:, 0], y0[:, -1], y0[:, :, 0], y0[:, :, -1] = 0, 0, 0, 0, 0, 0
    f = np.zeros_like(y0)
    for n in (1, 4):
        got = oracle.rbgs(y0, f, 1.0 / 8, n)
        assert np.max(np.abs(got - mu ** (2 * n) * y0)) <= 1e-13 * np.max(np.abs(y0)), (n, mu)


def test_exact_solution_fixed_point_and_convergence():
    nx, ny, nz = 10, 8, 12
    h = 1.0 / 11
    rng = np.random.default_rng(5)
    f = np.zeros((nz + 2, ny + 2, nx + 2))
    f[1:-1, 1:-1, 1:-1] = rng.standard_normal((nz, ny, nx))
    ud = exact.solve(f, h)
    got = oracle.rbgs(ud, f, h, 1)
    assert np.max(np.abs(got - ud)) <= 1e-13 * np.max(np.abs(ud))
    u = oracle.rbgs(np.zeros_like(f), f, h, 400)
    assert np.max(np.abs(u - ud)) <= 1e-9 * np.max(np.abs(ud))
    # red-black converges faster than Jacobi over the same number of sweeps
    uj = oracle.jacobi(np.zeros_like(f), f, h, 60)
    ur = oracle.rbgs(np.zeros_like(f), f, h, 60)
    assert np.max(np.abs(ur - ud)) < 0.5 * np.max(np.abs(uj - ud))


def test_low_precision_variants_follow_fp64():
    nx, ny, nz = 12, 9, 7
    rng = np.random.default_rng(8)
    u = rng.random((nz + 2, ny + 2, nx + 2))
    f = rng.standard_normal(u.shape)
    h = 1.0 / 13
    ref = oracle.rbgs(u, f, h, 2)
    g32 = oracle.rbgs_f32(u.astype(np.float32), f.astype(np.float32), h, 2)
    assert np.max(np.abs(g32 - ref)) <= 1e-6 * np.max(np.abs(ref))
    u16, f16 = oracle.to_bf16(u.astype(np.float32)), oracle.to_bf16(f.astype(np.float32))
    g16 = oracle.from_bf16(oracle.rbgs_bf16(u16, f16, h, 2))
    assert np.max(np.abs(g16 - ref)) <= 2 ** -6 * np.max(np.abs(ref))
