"""Closed-form discrete Poisson solution (test infrastructure only).

The 7-point operator A = (6 I - neighbour sum)/h^2 with zero Dirichlet halo
is diagonalised by the type-I discrete sine transform: the eigenvector
sin(pi p i/(nx+1)) sin(pi q j/(ny+1)) sin(pi r k/(nz+1)) has eigenvalue
    lambda = (2/h^2) * sum_d (1 - cos theta_d),  theta_d = pi p_d/(n_d+1).
So A^{-1} f = DST^{-1}(DST(f) / lambda).  scipy's orthonormal DST-I is its
own inverse.  Used to pin the sweep (its fixed point) and the residual.
"""
import numpy as np
from scipy.fft import dstn


def _half_angles(nx, ny, nz):
    """theta_d / 2 = pi p_d / (2 (n_d + 1)) per axis, broadcast (z, y, x)."""
    def ax(n):
        return np.pi * np.arange(1, n + 1, dtype=np.float64) / (2 * (n + 1))
    return ax(nz)[:, None, None], ax(ny)[None, :, None], ax(nx)[None, None, :]


def eigenvalues(nx, ny, nz, h):
    """lambda = (2/h^2) sum_d (1 - cos theta_d), with 1 - cos theta written
    2 sin^2(theta/2): the same value without the cancellation that costs the
    smoothest modes their relative accuracy on large grids."""
    az, ay, ax = _half_angles(nx, ny, nz)
    return (2.0 / (h * h)) * (2.0 * np.sin(az) ** 2 + 2.0 * np.sin(ay) ** 2 + 2.0 * np.sin(ax) ** 2)


def solve(f, h):
    """Exact discrete solution of A u = f with zero halo; f halo-shaped."""
    f = np.asarray(f, dtype=np.float64)
    nz, ny, nx = (s - 2 for s in f.shape)
    fi = f[1:-1, 1:-1, 1:-1]
    c = dstn(fi, type=1, norm="ortho")
    u = np.zeros_like(f)
    u[1:-1, 1:-1, 1:-1] = dstn(c / eigenvalues(nx, ny, nz, h), type=1, norm="ortho")
    return u


def jacobi_sweeps(u0, f, h, nsweeps):
    """The result of nsweeps Jacobi sweeps of the 7-point Poisson relaxation
    (Section 4.1, in the Poisson form u' = (six neighbours + h^2 f) / 6)
    from u0, with a zero Dirichlet halo, in closed form.  The sweep is
    u' = J u + (h^2 / 6) f with J = I - (h^2 / 6) A, so in the sine basis
    every mode evolves on its own: J's eigenvalue is
    mu = (cos theta_x + cos theta_y + cos theta_z) / 3 = 1 - (h^2 / 6) lambda,
    and after n sweeps
        u_n = mu^n (u0 - f / lambda) + f / lambda    (coefficient-wise).
    mu^n = sign^n exp(n log|mu|), with log|mu| = log1p(-(1 - |mu|)) and
    1 - |mu| formed without cancellation: (1/3) sum 2 sin^2(theta/2) where
    mu >= 0, (1/3) sum 2 cos^2(theta/2) where mu < 0 (a mode with mu near 1
    otherwise loses about n ulps of mu^n).  Exact up to the transforms'
    rounding; u0 and f halo-shaped, their halos zero."""
    u0 = np.asarray(u0, dtype=np.float64)
    f = np.asarray(f, dtype=np.float64)
    nz, ny, nx = (s - 2 for s in u0.shape)
    az, ay, ax = _half_angles(nx, ny, nz)
    one_minus = (2.0 * np.sin(az) ** 2 + 2.0 * np.sin(ay) ** 2 + 2.0 * np.sin(ax) ** 2) / 3.0  # 1 - mu
    one_plus = (2.0 * np.cos(az) ** 2 + 2.0 * np.cos(ay) ** 2 + 2.0 * np.cos(ax) ** 2) / 3.0   # 1 + mu
    lam = (6.0 / (h * h)) * one_minus
    nonneg = one_minus <= 1.0
    with np.errstate(divide="ignore"):
        log_abs = np.where(nonneg, np.log1p(-np.minimum(one_minus, 1.0)), np.log1p(-np.minimum(one_plus, 1.0)))
    mun = np.exp(nsweeps * log_abs)
    if nsweeps % 2:
        mun = np.where(nonneg, mun, -mun)
    fs = dstn(f[1:-1, 1:-1, 1:-1], type=1, norm="ortho") / lam
    us = dstn(u0[1:-1, 1:-1, 1:-1], type=1, norm="ortho")
    out = np.zeros_like(u0)
    out[1:-1, 1:-1, 1:-1] = dstn(mun * (us - fs) + fs, type=1, norm="ortho")
    return out
