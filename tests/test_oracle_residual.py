"""Pins for the oracle's FP64 residual r = f - A u (A the 7-point operator
(6u - neighbour sum)/h^2) and its norms."""
import numpy as np

import oracle
from oracle import exact
from paper_2310_01882_b300 import inputs
from tests.test_oracle_jacobi import dense_system, sss


def test_residual_of_exact_solution_vanishes():
    n = 12
    f = inputs.grf(n, seed=11)
    h = 1.0 / (n + 1)
    ud = exact.solve(f, h)
    nr, nf = oracle.residual(ud, f, h)
    assert nr <= 1e-12 * nf


def test_residual_of_zero_is_f():
    n = 9
    f = inputs.grf(n, seed=12)
    nr, nf, r = oracle.residual(np.zeros_like(f), f, 1.0 / (n + 1), want_r=True)
    assert nr == nf
    assert np.array_equal(r[1:-1, 1:-1, 1:-1], f[1:-1, 1:-1, 1:-1])
    assert abs(nf - np.sqrt(np.sum(f[1:-1, 1:-1, 1:-1] ** 2))) <= 1e-14 * nf


def test_eigenvector_closed_form():
    """A SSS = lambda_h SSS with lambda_h = (2/h^2) sum_d (1 - cos(m_d pi/(n_d+1)))."""
    nx, ny, nz = 11, 8, 6
    h = 0.05
    u = sss(nx, ny, nz, 2, 1, 3)
    lam = (2 / h ** 2) * ((1 - np.cos(2 * np.pi / (nx + 1))) + (1 - np.cos(np.pi / (ny + 1)))
                          + (1 - np.cos(3 * np.pi / (nz + 1))))
    f = np.zeros_like(u)
    _, _, r = oracle.residual(u, f, h, want_r=True)
    assert np.max(np.abs(r + lam * u)) <= 1e-12 * lam


def test_linearity():
    rng = np.random.default_rng(2)
    shape = (7, 6, 9)
    u1, u2, f1, f2 = (rng.standard_normal(shape) for _ in range(4))
    h = 0.1
    _, _, r1 = oracle.residual(u1, f1, h, want_r=True)
    _, _, r2 = oracle.residual(u2, f2, h, want_r=True)
    _, _, r12 = oracle.residual(u1 + u2, f1 + f2, h, want_r=True)
    assert np.max(np.abs(r12 - r1 - r2)) <= 1e-12 * np.max(np.abs(r12))


def test_brute_force_4cubed():
    """r = f - A u with A from the dense neighbour relation: the sweep's
    affine map x' = M x + c satisfies A x = (6/h^2)(x - M x) - (6/h^2)(c - h^2 f/6)."""
    rng = np.random.default_rng(7)
    n = 4
    h = 0.25
    u = rng.random((n + 2,) * 3)
    f = rng.standard_normal((n + 2,) * 3)
    M, c, pts = dense_system(n, n, n, h, np.zeros_like(f), u)  # c = halo terms / 6
    x = np.array([u[k, j, i] for (i, j, k) in pts])
    fx = np.array([f[k, j, i] for (i, j, k) in pts])
    Ax = (6.0 / h ** 2) * (x - M @ x - c)
    nr, nf, r = oracle.residual(u, f, h, want_r=True)
    got = np.array([r[k, j, i] for (i, j, k) in pts])
    np.testing.assert_allclose(got, fx - Ax, rtol=0, atol=1e-12 * np.max(np.abs(Ax)))
    assert abs(nr - np.linalg.norm(fx - Ax)) <= 1e-12 * nr
    assert abs(nf - np.linalg.norm(fx)) <= 1e-14 * nf
