"""Closed-form discrete Poisson solution (test infrastructure only).

The 7-point operator A = (6 I - neighbour sum)/h^2 with zero Dirichlet halo
is diagonalised by the type-I discrete sine transform: the eigenvector
sin(pi p i/(nx+1)) sin(pi q j/(ny+1)) sin(pi r k/(nz+1)) has eigenvalue
    lambda = (2/h^2) * sum_d (1 - cos(pi p_d/(n_d+1))).
So A^{-1} f = DST^{-1}(DST(f) / lambda).  scipy's orthonormal DST-I is its
own inverse.  Used to pin the sweep (its fixed point) and the residual.
"""
import numpy as np
from scipy.fft import dstn


def eigenvalues(nx, ny, nz, h):
    def ax(n):
        p = np.arange(1, n + 1, dtype=np.float64)
        return 1.0 - np.cos(np.pi * p / (n + 1))
    lx, ly, lz = ax(nx), ax(ny), ax(nz)
    return (2.0 / (h * h)) * (lz[:, None, None] + ly[None, :, None] + lx[None, None, :])


def solve(f, h):
    """Exact discrete solution of A u = f with zero halo; f halo-shaped."""
    f = np.asarray(f, dtype=np.float64)
    nz, ny, nx = (s - 2 for s in f.shape)
    fi = f[1:-1, 1:-1, 1:-1]
    c = dstn(fi, type=1, norm="ortho")
    u = np.zeros_like(f)
    u[1:-1, 1:-1, 1:-1] = dstn(c / eigenvalues(nx, ny, nz, h), type=1, norm="ortho")
    return u
