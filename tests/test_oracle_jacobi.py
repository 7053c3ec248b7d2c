"""Pins for the oracle's Jacobi sweep (Section 4.1's 7-point relaxation,
Poisson form).  Each pin is fixed by the mathematics, not by re-typing the
sweep: an eigenvector identity, an exact fixed point, O(h^2) convergence to the
continuum solution, a dense matrix built from the neighbour relation, and the
DST closed-form solution."""
import numpy as np
import pytest

import oracle
from oracle import exact
from paper_2310_01882_b300 import inputs


def sss(nx, ny, nz, p=1, q=1, r=1):
    """sin(p pi i/(nx+1)) sin(q pi j/(ny+1)) sin(r pi k/(nz+1)), zero halo."""
    def ax(n, m):
        i = np.arange(n + 2, dtype=np.float64)
        s = np.sin(m * np.pi * i / (n + 1))
        s[0] = 0.0
        s[-1] = 0.0
        return s
    return ax(nz, r)[:, None, None] * ax(ny, q)[None, :, None] * ax(nx, p)[None, None, :]


def test_discrete_fixed_point():
    """u_d = 3 pi^2 / lambda_h * SSS solves A u = 3 pi^2 SSS exactly, so one
    sweep maps it to itself (lambda_h = 12 sin^2(pi h/2)/h^2)."""
    n = 24
    f, h = inputs.sin_source(n)
    lam = 12.0 * np.sin(np.pi * h / 2) ** 2 / h ** 2
    ud = 3.0 * np.pi ** 2 / lam * sss(n, n, n)
    out = oracle.jacobi_sweep(ud, f, h)
    assert np.max(np.abs(out - ud)) <= 8 * np.finfo(float).eps * np.max(np.abs(ud))


@pytest.mark.parametrize("pqr", [(1, 2, 3), (3, 1, 2), (5, 4, 1)])
def test_mode_decay(pqr):
    """With f = 0 a separable sine mode is an eigenvector of the sweep with
    eigenvalue mu = (cos(p pi/(nx+1)) + cos(q pi/(ny+1)) + cos(r pi/(nz+1)))/3.
    Distinct extents per axis catch a transposed index."""
    nx, ny, nz = 13, 9, 6
    p, q, r = pqr
    e0 = sss(nx, ny, nz, p, q, r)
    mu = (np.cos(p * np.pi / (nx + 1)) + np.cos(q * np.pi / (ny + 1)) + np.cos(r * np.pi / (nz + 1))) / 3
    f = np.zeros_like(e0)
    for k in (1, 10, 100):
        ek = oracle.jacobi(e0, f, 0.1, k)
        assert np.max(np.abs(ek - mu ** k * e0)) <= 1e-13 * max(abs(mu) ** k, 1e-3)


def test_second_order_convergence():
    """Iterating to convergence from zero reproduces the continuum solution
    sin sin sin of -Lap u = 3 pi^2 sin sin sin with error O(h^2)."""
    errs = []
    for n in (7, 15, 31):
        f, h = inputs.sin_source(n)
        sweeps = int(4.0 * (n + 1) ** 2 * np.log(1e13) / np.pi ** 2) + 10
        u = oracle.jacobi(np.zeros_like(f), f, h, sweeps, nthreads=0)
        errs.append(np.max(np.abs(u - sss(n, n, n))))
    ratios = [errs[i] / errs[i + 1] for i in range(2)]
    for rt in ratios:
        assert 3.6 < rt < 4.4, (errs, ratios)


def dense_system(nx, ny, nz, h, f, halo_u):
    """Build the sweep as x' = M x + c from the neighbour relation alone:
    M[p, q] = 1/6 for each interior neighbour q of interior point p;
    c[p] = (h^2 f[p] + sum of halo-neighbour values)/6."""
    pts = [(i, j, k) for k in range(1, nz + 1) for j in range(1, ny + 1) for i in range(1, nx + 1)]
    index = {pt: n for n, pt in enumerate(pts)}
    N = len(pts)
    M = np.zeros((N, N))
    c = np.zeros(N)
    for n, (i, j, k) in enumerate(pts):
        c[n] += h * h * f[k, j, i]
        for d in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
            nb = (i + d[0], j + d[1], k + d[2])
            if nb in index:
                M[n, index[nb]] += 1.0
            else:
                c[n] += halo_u[nb[2], nb[1], nb[0]]
    return M / 6.0, c / 6.0, pts


def test_brute_force_4cubed():
    """One sweep on 4^3 (random interior and random nonzero halo) equals the
    dense affine map built from the neighbour relation; the dense solution of
    A u = f is a fixed point of the sweep; out's halo is u's halo."""
    rng = np.random.default_rng(0)
    n = 4
    u = rng.random((n + 2,) * 3)
    f = rng.standard_normal((n + 2,) * 3)
    h = 0.2
    M, c, pts = dense_system(n, n, n, h, f, u)
    x = np.array([u[k, j, i] for (i, j, k) in pts])
    out = oracle.jacobi_sweep(u, f, h)
    got = np.array([out[k, j, i] for (i, j, k) in pts])
    np.testing.assert_allclose(got, M @ x + c, rtol=0, atol=1e-15 * np.max(np.abs(got)) * 8)
    inner = np.zeros((n + 2,) * 3, dtype=bool)
    inner[1:-1, 1:-1, 1:-1] = True
    assert np.array_equal(out[~inner], u[~inner])
    # fixed point: (I - M) x* = c
    xs = np.linalg.solve(np.eye(len(pts)) - M, c)
    us = u.copy()
    for val, (i, j, k) in zip(xs, pts):
        us[k, j, i] = val
    out2 = oracle.jacobi_sweep(us, f, h)
    assert np.max(np.abs(out2 - us)) <= 1e-14 * np.max(np.abs(us))


def test_converges_to_dst_solution():
    """Jacobi iterates converge to the closed-form (DST-I) discrete solution."""
    n = 8
    f = inputs.grf(n, seed=5)
    h = 1.0 / (n + 1)
    ud = exact.solve(f, h)
    u = oracle.jacobi(np.zeros_like(f), f, h, 3000)
    assert np.max(np.abs(u - ud)) <= 1e-12 * np.max(np.abs(ud))


def test_f32_sweep_within_fp32_bound():
    """FP32 storage + arithmetic sweep agrees with the FP64 sweep of the same
    FP32-rounded inputs to within a few FP32 roundings of the largest term."""
    rng = np.random.default_rng(3)
    u = rng.random((10, 9, 12)).astype(np.float32)
    f = rng.standard_normal((10, 9, 12)).astype(np.float32)
    h = 1.0 / 11
    o32 = oracle.jacobi_sweep_f32(u, f, h)
    o64 = oracle.jacobi_sweep(u.astype(np.float64), f.astype(np.float64), np.float64(oracle.f32_coeff(h)) ** 0.5)
    err = np.max(np.abs(o32.astype(np.float64) - o64)) / np.max(np.abs(o64))
    assert err < 8 * 2.0 ** -24


def test_bf16_rounding_matches_torch():
    """The bf16 rounding is IEEE round-to-nearest-even of the upper 16 bits:
    it agrees bit for bit with torch's float32 -> bfloat16 conversion,
    including ties (1 + 2^-8 rounds to 1, 1 + 3*2^-8 rounds up)."""
    import torch
    rng = np.random.default_rng(1)
    x = np.concatenate([rng.standard_normal(10000).astype(np.float32),
                        np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -0.0, 65504.0, 1e-40], np.float32)])
    ours = oracle.to_bf16(x)
    theirs = torch.from_numpy(x).to(torch.bfloat16).view(torch.int16).numpy().view(np.uint16)
    assert np.array_equal(ours, theirs)
    assert ours[-5] == 0x3F80 and ours[-4] == 0x3F82
    back = oracle.from_bf16(ours)
    assert np.array_equal(back, torch.from_numpy(x).to(torch.bfloat16).float().numpy())


def test_bf16_sweep_within_bf16_bound():
    rng = np.random.default_rng(4)
    u = rng.random((8, 8, 8)).astype(np.float32)
    f = rng.standard_normal((8, 8, 8)).astype(np.float32)
    h = 1.0 / 7
    u16, f16 = oracle.to_bf16(u), oracle.to_bf16(f)
    o16 = oracle.from_bf16(oracle.jacobi_sweep_bf16(u16, f16, h)).astype(np.float64)
    o64 = oracle.jacobi_sweep(oracle.from_bf16(u16).astype(np.float64),
                              oracle.from_bf16(f16).astype(np.float64), h)
    assert np.max(np.abs(o16 - o64)) / np.max(np.abs(o64)) <= 2.0 ** -8


@pytest.mark.parametrize("nsweeps", [0, 1, 7, 60])
def test_closed_form_sweeps_match_the_loops(nsweeps):
    """exact.jacobi_sweeps (the sweep's modal closed form) equals nsweeps
    sweeps of the loop oracle on a non-cubic grid with a random start and
    source (zero halo)."""
    nx, ny, nz = 13, 9, 11
    rng = np.random.default_rng(40 + nsweeps)
    u0 = np.zeros((nz + 2, ny + 2, nx + 2))
    u0[1:-1, 1:-1, 1:-1] = rng.random((nz, ny, nx))
    f = np.zeros_like(u0)
    f[1:-1, 1:-1, 1:-1] = rng.standard_normal((nz, ny, nx))
    h = 1.0 / 14
    ref = oracle.jacobi(u0, f, h, nsweeps)
    got = exact.jacobi_sweeps(u0, f, h, nsweeps)
    assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))


def test_closed_form_sweeps_mode_and_limit():
    """A single sine mode with f = 0 decays by mu^n; with a source, many
    sweeps approach the discrete solution."""
    nx, ny, nz = 10, 7, 12
    h = 1.0 / 13
    e0 = sss(nx, ny, nz, 2, 1, 3)
    mu = (np.cos(2 * np.pi / (nx + 1)) + np.cos(np.pi / (ny + 1)) + np.cos(3 * np.pi / (nz + 1))) / 3
    got = exact.jacobi_sweeps(e0, np.zeros_like(e0), h, 25)
    assert np.max(np.abs(got - mu ** 25 * e0)) <= 1e-14
    f = inputs.grf(nx, seed=8, ny=ny, nz=nz)
    far = exact.jacobi_sweeps(np.zeros_like(f), f, h, 100000)
    ud = exact.solve(f, h)
    assert np.max(np.abs(far - ud)) <= 1e-12 * np.max(np.abs(ud))
