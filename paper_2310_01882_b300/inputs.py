"""Seeded synthetic inputs shaped like the paper's benchmarks.

This module only draws and shapes random data; it holds none of the stencil
arithmetic.  Both the CUDA path and the CPU oracle are fed from it.  Every
field is a numpy array of shape (nz+2, ny+2, nx+2), x fastest, with a
one-cell halo (the caller's boundary values).

Recipes:
  * sin_source:   f = 3 pi^2 sin(pi x) sin(pi y) sin(pi z) at x = i h,
                  h = 1/(n+1) (the manufactured solution sin*sin*sin).
  * uniform:      iid U[0,1) on the interior, zero halo.
  * grf:          Gaussian random field with power spectrum ~ |k|^-3: iid
                  N(0,1) coefficients on the sine modes k in {1..n}^3 scaled
                  by |k|^(-3/2), sent through an orthonormal DST-I (so the
                  field vanishes on the Dirichlet boundary) and normalised to
                  unit RMS.
  * winds:        u, v, w each a sum of 8 sinusoids
                  A sin(2 pi (kx x/Nx + ky y/Ny + kz z/Nz) + phi), integer
                  kx, ky in [1, 8] (periodic in x and y), kz in [0, 4],
                  phi ~ U[0, 2 pi), A = 10/sqrt(8) (RMS ~ 7 m/s, peaks ~10),
                  plus N(0, 0.1) noise; halos periodic in x, y and zero in z.
  * tzc:          vertical factors U[0.5, 1.5) of length nz.
"""
import numpy as np
from scipy.fft import dstn


def grid_coords(n):
    """x_i = i h for halo-inclusive indices i = 0..n+1, h = 1/(n+1)."""
    h = 1.0 / (n + 1)
    return np.arange(n + 2, dtype=np.float64) * h, h


def sin_source(n):
    """f = 3 pi^2 S(x)S(y)S(z), S = sin(pi .), on an n^3 grid; returns (f, h)."""
    x, h = grid_coords(n)
    s = np.sin(np.pi * x)
    s[0] = 0.0
    s[-1] = 0.0
    f = 3.0 * np.pi ** 2 * s[:, None, None] * s[None, :, None] * s[None, None, :]
    return f, h


def uniform(nx, ny, nz, seed):
    """iid U[0,1) interior, zero halo."""
    rng = np.random.default_rng(seed)
    a = np.zeros((nz + 2, ny + 2, nx + 2), dtype=np.float64)
    a[1:-1, 1:-1, 1:-1] = rng.random((nz, ny, nx))
    return a


def grf(n, seed, ny=None, nz=None):
    """k^-3 Gaussian random field, zero halo, unit RMS interior."""
    nx = n
    ny = n if ny is None else ny
    nz = n if nz is None else nz
    rng = np.random.default_rng(seed)
    kz = np.arange(1, nz + 1, dtype=np.float64)[:, None, None]
    ky = np.arange(1, ny + 1, dtype=np.float64)[None, :, None]
    kx = np.arange(1, nx + 1, dtype=np.float64)[None, None, :]
    amp = (kx * kx + ky * ky + kz * kz) ** (-0.75)
    c = rng.standard_normal((nz, ny, nx)) * amp
    field = dstn(c, type=1, norm="ortho")
    field /= np.sqrt(np.mean(field * field))
    a = np.zeros((nz + 2, ny + 2, nx + 2), dtype=np.float64)
    a[1:-1, 1:-1, 1:-1] = field
    return a


def fill_periodic_xy(a):
    """Copy interior edges into the x and y halo (periodic), in place."""
    a[:, :, 0] = a[:, :, -2]
    a[:, :, -1] = a[:, :, 1]
    a[:, 0, :] = a[:, -2, :]
    a[:, -1, :] = a[:, 1, :]
    return a


def wind(nx, ny, nz, seed, terms=8, amplitude=10.0, noise=0.1):
    """One velocity component: random-phase sinusoids + noise, periodic x, y."""
    rng = np.random.default_rng(seed)
    A = amplitude / np.sqrt(terms)
    z = np.arange(nz, dtype=np.float64)[:, None, None]
    y = np.arange(ny, dtype=np.float64)[None, :, None]
    x = np.arange(nx, dtype=np.float64)[None, None, :]
    field = np.zeros((nz, ny, nx), dtype=np.float64)
    for _ in range(terms):
        kx = rng.integers(1, 9)
        ky = rng.integers(1, 9)
        kz = rng.integers(0, 5)
        phi = rng.random() * 2.0 * np.pi
        field += A * np.sin(2.0 * np.pi * (kx * x / nx + ky * y / ny + kz * z / nz) + phi)
    field += rng.normal(0.0, noise, size=(nz, ny, nx))
    a = np.zeros((nz + 2, ny + 2, nx + 2), dtype=np.float64)
    a[1:-1, 1:-1, 1:-1] = field
    return fill_periodic_xy(a)


def winds(nx, ny, nz, seeds=(4, 5, 6)):
    return tuple(wind(nx, ny, nz, s) for s in seeds)


def tzc(nz, seed):
    rng = np.random.default_rng(seed)
    return 0.5 + rng.random(nz)


def batch_sizes(count=256, lo=32, hi=192, seed=9):
    """Cubic instance sizes drawn uniform in [lo, hi]."""
    rng = np.random.default_rng(seed)
    return [int(s) for s in rng.integers(lo, hi + 1, size=count)]
