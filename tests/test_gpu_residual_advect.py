"""GPU parity of stencil_residual and stencil_advect_uvw."""
import numpy as np
import pytest

import oracle
from oracle import exact
from paper_2310_01882_b300 import inputs
from paper_2310_01882_b300 import stencil as S
from tests.gpu_util import ctx, rel_err

pytestmark = pytest.mark.gpu

SHAPES = [(64, 64, 64), (67, 35, 19), (1, 1, 1), (3, 130, 2), (130, 17, 70)]


def gpu_residual(u, f, h, want_r=True):
    import torch
    uf, ff = S.Field.from_numpy(u), S.Field.from_numpy(f)
    rf = S.Field(uf.nx, uf.ny, uf.nz) if want_r else None
    norms = torch.zeros(2, dtype=torch.float64, device="cuda")
    S.stencil_residual(ctx(), uf, ff, h, norms, r=rf)
    torch.cuda.synchronize()
    n = norms.cpu().numpy()
    return n[0], n[1], (rf.to_numpy() if want_r else None)


def r_tol(u, f, h):
    """Bound on |r_gpu - r_oracle| per point.  Both are within a few
    rounding units of the exact f - A u: the library's fixed-point
    evaluation within 6.5 units of 2^-S <= 2^-61 (12 max|u| + h^2 max|f|),
    divided by h^2 (plus the final rounding); the oracle's binary64
    evaluation in the written order within about 16 eps (12 max|u| / h^2 +
    max|f|).  1e-14 of that scale covers both."""
    return 1e-14 * (12.0 * np.max(np.abs(u)) / (h * h) + np.max(np.abs(f[1:-1, 1:-1, 1:-1])))


def check_residual(u, f, h):
    nr, nf, r = oracle.residual(u, f, h, want_r=True, nthreads=0)
    gr, gf, rg = gpu_residual(u, f, h)
    tol = r_tol(u, f, h)
    d = np.max(np.abs(rg[1:-1, 1:-1, 1:-1] - r[1:-1, 1:-1, 1:-1]))
    assert d <= tol, (d, tol)
    npts = r[1:-1, 1:-1, 1:-1].size
    assert abs(gr - nr) <= np.sqrt(npts) * tol + 1e-12 * nr, (gr, nr)
    assert abs(gf - nf) <= 1e-13 * nf
    gr2, _, _ = gpu_residual(u, f, h, want_r=False)
    assert gr2 == gr          # the same norm with or without r written
    return r, rg


@pytest.mark.parametrize("shape", SHAPES)
def test_residual_per_point(shape):
    nx, ny, nz = shape
    rng = np.random.default_rng(sum(shape))
    u = rng.random((nz + 2, ny + 2, nx + 2))
    f = rng.standard_normal((nz + 2, ny + 2, nx + 2))
    check_residual(u, f, 1.0 / (max(shape) + 1))


@pytest.mark.parametrize("shape", [(64, 64, 64), (67, 35, 19)])
def test_residual_near_convergence(shape):
    """u within 1e-9 of the discrete solution: r is a small difference of
    large terms, and both evaluations agree to their rounding bound."""
    nx, ny, nz = shape
    f = inputs.grf(nx, seed=5, ny=ny, nz=nz)
    h = 1.0 / (max(shape) + 1)
    ud = exact.solve(f, h)
    rng = np.random.default_rng(6)
    ud[1:-1, 1:-1, 1:-1] += 1e-9 * np.max(np.abs(ud)) * rng.standard_normal((nz, ny, nx))
    check_residual(ud, f, h)


def test_residual_unaligned_grid_is_bitwise():
    """A grid whose rows a TMA descriptor cannot address (odd row length in
    elements) takes the binary64 kernel: r bitwise the oracle's."""
    import torch
    nx, ny, nz = 13, 7, 5
    rng = np.random.default_rng(9)
    u = rng.random((nz + 2, ny + 2, nx + 2))
    f = rng.standard_normal(u.shape)
    h = 1.0 / 14
    sy = nx + 2                      # 15 doubles: rows not 16-byte aligned
    sz = sy * (ny + 2)

    def raw(a):
        t = torch.from_numpy(np.ascontiguousarray(a)).cuda()
        return t, S.stencil_grid(t.data_ptr(), nx, ny, nz, sy, sz, S.F64, 0)

    tu, gu = raw(u)
    tf, gf = raw(f)
    tr, gr = raw(np.zeros_like(u))
    norms = torch.zeros(2, dtype=torch.float64, device="cuda")
    import ctypes
    rc = S.lib().stencil_residual(ctx().handle, ctypes.byref(gu), ctypes.byref(gf), h, ctypes.byref(gr),
                                  ctypes.c_void_p(norms.data_ptr()), None)
    assert rc == 0
    torch.cuda.synchronize()
    nr, nf, r = oracle.residual(u, f, h, want_r=True)
    assert np.array_equal(tr.cpu().numpy()[1:-1, 1:-1, 1:-1], r[1:-1, 1:-1, 1:-1])
    assert abs(norms[0].item() - nr) <= 1e-13 * nr


def test_residual_deterministic_and_exact_solution():
    n = 48
    f = inputs.grf(n, seed=31)
    h = 1.0 / (n + 1)
    ud = exact.solve(f, h)
    a = gpu_residual(ud, f, h, want_r=False)
    b = gpu_residual(ud, f, h, want_r=False)
    assert a[0] == b[0] and a[1] == b[1]
    assert a[0] <= 1e-12 * a[1]


def test_residual_scale_follows_each_input():
    """The fixed-point residual's scale comes from the magnitudes of what its
    pass reads.  A context reuses the previous call's magnitudes as the
    guess and repeats the pass when the guess gives another scale.  On one
    context, fields of very different magnitudes in turn (1e-120, 1e+120,
    1, 1 again, 1e-120 again) each match the oracle, and every call returns
    bit for bit what a fresh context's first call returns for the same
    input, so the result does not depend on what ran before."""
    import torch
    from paper_2310_01882_b300.stencil import Context
    nx, ny, nz = 45, 30, 21
    rng = np.random.default_rng(77)
    base_u = rng.random((nz + 2, ny + 2, nx + 2))
    base_f = rng.standard_normal((nz + 2, ny + 2, nx + 2))
    h = 1.0 / 46
    shared = Context(0)

    def run(c, u, f):
        uf, ff = S.Field.from_numpy(u), S.Field.from_numpy(f)
        rf = S.Field(nx, ny, nz)
        norms = torch.zeros(2, dtype=torch.float64, device="cuda")
        S.stencil_residual(c, uf, ff, h, norms, r=rf)
        torch.cuda.synchronize()
        S.stencil_ctx_status(c)
        return norms.cpu().numpy(), rf.to_numpy()

    for scale in (1e-120, 1e120, 1.0, 1.0, 1e-120):
        u, f = scale * base_u, scale * base_f
        nr, nf, r = oracle.residual(u, f, h, want_r=True, nthreads=0)
        got_n, got_r = run(shared, u, f)
        tol = r_tol(u, f, h)
        assert np.max(np.abs(got_r[1:-1, 1:-1, 1:-1] - r[1:-1, 1:-1, 1:-1])) <= tol
        assert abs(got_n[0] - nr) <= np.sqrt(nx * ny * nz) * tol + 1e-12 * nr
        assert abs(got_n[1] - nf) <= 1e-13 * nf
        fresh = Context(0)
        ref_n, ref_r = run(fresh, u, f)
        fresh.close()
        assert np.array_equal(got_n, ref_n) and np.array_equal(got_r, ref_r), scale
    shared.close()


def test_residual_nonfinite_then_finite():
    """A NaN (or an infinity) in u: the fixed-point residual's norms are NaN
    and the context reports STENCIL_ERR_NONFINITE; the next call on the same
    context, with finite input, is right again (its scale guess recovers)."""
    import torch
    from paper_2310_01882_b300.stencil import Context
    n = 20
    rng = np.random.default_rng(81)
    u = rng.random((n + 2, n + 2, n + 2))
    f = rng.standard_normal((n + 2, n + 2, n + 2))
    h = 1.0 / (n + 1)
    c = Context(0)
    norms = torch.zeros(2, dtype=torch.float64, device="cuda")
    for bad in (np.nan, np.inf):
        ub = u.copy()
        ub[7, 8, 9] = bad
        S.stencil_residual(c, S.Field.from_numpy(ub), S.Field.from_numpy(f), h, norms)
        torch.cuda.synchronize()
        assert np.isnan(norms.cpu().numpy()).all()
        with pytest.raises(S.StencilError) as e:
            S.stencil_ctx_status(c)
        assert e.value.code == -6
        S.stencil_ctx_status(c)  # cleared
        S.stencil_residual(c, S.Field.from_numpy(u), S.Field.from_numpy(f), h, norms)
        torch.cuda.synchronize()
        S.stencil_ctx_status(c)
        nr, nf = oracle.residual(u, f, h)
        g = norms.cpu().numpy()
        assert abs(g[0] - nr) <= 1e-12 * nr and abs(g[1] - nf) <= 1e-13 * nf
    c.close()


def test_residual_full_size_norms():
    """512^3 with the benchmark's source (k^-3 field) and a U[0,1) iterate:
    norms agree with the oracle's (all host cores)."""
    n = 512
    f = inputs.grf(n, seed=2)
    u = inputs.uniform(n, n, n, seed=3)
    h = 1.0 / (n + 1)
    nr, nf = oracle.residual(u, f, h, nthreads=0)
    gr, gf, _ = gpu_residual(u, f, h, want_r=False)
    assert abs(gr - nr) <= 1e-12 * nr and abs(gf - nf) <= 1e-12 * nf


def run_advect(u, v, w, t1, t2, tcx=0.25, tcy=0.25):
    import torch
    fu, fv, fw = (S.Field.from_numpy(a) for a in (u, v, w))
    su, sv, sw = fu.like(), fu.like(), fu.like()
    d1 = torch.from_numpy(np.ascontiguousarray(t1)).cuda()
    d2 = torch.from_numpy(np.ascontiguousarray(t2)).cuda()
    S.stencil_advect_uvw(ctx(), fu, fv, fw, su, sv, sw, d1, d2, tcx, tcy)
    torch.cuda.synchronize()
    return su.to_numpy(), sv.to_numpy(), sw.to_numpy()


@pytest.mark.parametrize("shape", SHAPES + [(512, 512, 16)])
def test_advect_parity(shape):
    nx, ny, nz = shape
    u, v, w = inputs.winds(nx, ny, nz, seeds=(4, 5, 6))
    t1, t2 = inputs.tzc(nz, 7), inputs.tzc(nz, 8)
    ref = oracle.advect_uvw(u, v, w, t1, t2, 0.25, 0.25)
    got = run_advect(u, v, w, t1, t2)
    for g, r in zip(got, ref):
        assert rel_err(g, r) <= 1e-13


def test_advect_every_config():
    """Each compiled tile configuration of the fixed-point kernel (pinned
    with advect_config_select) matches the oracle: ragged x/y tiles, several
    z chunks, tcy not a power of two (the multiplied factor path) and a
    power of two (the shifted one)."""
    import torch
    from paper_2310_01882_b300.stencil import Context
    count = S.stencil_advect_config_count()
    assert count >= 1
    nx, ny, nz = 45, 37, 70
    u, v, w = inputs.winds(nx, ny, nz, seeds=(41, 42, 43))
    t1, t2 = inputs.tzc(nz, 7), inputs.tzc(nz, 8)
    d1, d2 = torch.from_numpy(t1).cuda(), torch.from_numpy(t2).cuda()
    fu, fv, fw = (S.Field.from_numpy(a) for a in (u, v, w))
    for tcy in (0.25, 0.3):
        ref = oracle.advect_uvw(u, v, w, t1, t2, 0.25, tcy)
        for idx in range(count):
            c = Context(0)
            S.stencil_advect_config_select(c, idx)
            outs = [fu.like() for _ in range(3)]
            S.stencil_advect_uvw(c, fu, fv, fw, *outs, d1, d2, 0.25, tcy)
            torch.cuda.synchronize()
            for o, r in zip(outs, ref):
                assert rel_err(o.to_numpy(), r) <= 1e-13, (idx, tcy)
            with pytest.raises(S.StencilError):
                S.stencil_advect_config_select(c, count)
            c.close()


def test_advect_scales_follow_each_input():
    """The advection's scales (and its choice between fixed point and
    binary64) come from the magnitudes of what its pass reads, the fields'
    and the factors'.  A context reuses the previous call's magnitudes as
    the guess and repeats the pass when the guess leads elsewhere.  On one
    context, winds scaled by 1e-150, 1e+150, 1, 1 again, then uneven
    magnitudes (w times 1e-7: binary64), then 1 again, then factors tzc1,
    tzc2 scaled by 2^-40 (another factor scale), factors of uneven
    magnitudes (tzc1 times 1e-5: binary64), the first factors again, and
    tcy = 0.3 (multiplied, not shifted) each match the oracle and equal bit
    for bit a fresh context's first call on the same input."""
    import torch
    from paper_2310_01882_b300.stencil import Context
    nx, ny, nz = 37, 29, 13
    u0, v0, w0 = inputs.winds(nx, ny, nz, seeds=(51, 52, 53))
    t10, t20 = inputs.tzc(nz, 7), inputs.tzc(nz, 8)
    shared = Context(0)

    def go(c, u, v, w, t1, t2, tcy):
        fu, fv, fw = (S.Field.from_numpy(a) for a in (u, v, w))
        d1, d2 = torch.from_numpy(t1).cuda(), torch.from_numpy(t2).cuda()
        outs = [fu.like() for _ in range(3)]
        S.stencil_advect_uvw(c, fu, fv, fw, *outs, d1, d2, 0.25, tcy)
        torch.cuda.synchronize()
        return [o.to_numpy() for o in outs]

    cases = ("tiny", "huge", "one", "one", "uneven", "one", "tzc_small", "tzc_uneven", "one", "tcy", "one")
    for case in cases:
        sc = {"tiny": 1e-150, "huge": 1e150}.get(case, 1.0)
        u, v, w = sc * u0, sc * v0, sc * w0
        if case == "uneven":
            w = 1e-7 * w
        t1, t2 = t10, t20
        if case == "tzc_small":
            t1, t2 = t10 * 2.0 ** -40, t20 * 2.0 ** -40
        elif case == "tzc_uneven":
            t1 = t10 * 1e-5
        tcy = 0.3 if case == "tcy" else 0.25
        ref = oracle.advect_uvw(u, v, w, t1, t2, 0.25, tcy)
        got = go(shared, u, v, w, t1, t2, tcy)
        for g, r in zip(got, ref):
            assert rel_err(g, r) <= 1e-13, case
        fresh = Context(0)
        again = go(fresh, u, v, w, t1, t2, tcy)
        fresh.close()
        for g, a in zip(got, again):
            assert np.array_equal(g, a), case
    shared.close()


def test_advect_full_size():
    """512 x 512 x 256, winds per the benchmark recipe, oracle on all cores;
    every compiled tile shape (at this size each keeps its own z chunk
    length); the default shape twice on one context, as the benchmark
    times it.  The normwise error is taken on the GPU (binary64)."""
    import torch
    from paper_2310_01882_b300.stencil import Context
    u, v, w = inputs.winds(512, 512, 256)
    t1, t2 = inputs.tzc(256, 7), inputs.tzc(256, 8)
    ref = [torch.from_numpy(r[1:-1, 1:-1, 1:-1].copy()).cuda()
           for r in oracle.advect_uvw(u, v, w, t1, t2, 0.25, 0.25, nthreads=0)]
    fu, fv, fw = (S.Field.from_numpy(a) for a in (u, v, w))
    d1, d2 = torch.from_numpy(t1).cuda(), torch.from_numpy(t2).cuda()
    outs = [fu.like() for _ in range(3)]
    for idx in range(S.stencil_advect_config_count()):
        c = Context(0)
        S.stencil_advect_config_select(c, idx)
        for call in range(2 if idx == 0 else 1):
            for o in outs:
                o.cells.fill_(float("nan"))
            S.stencil_advect_uvw(c, fu, fv, fw, *outs, d1, d2, 0.25, 0.25)
            for o, r in zip(outs, ref):
                err = ((o.cells[1:-1, 1:-1, 1:-1] - r).abs().max() / r.abs().max()).item()
                assert err <= 1e-13, (idx, call, err)
        c.close()


def test_advect_constant_fields_zero():
    """Constant fields with tzc1 = tzc2: the tendency is exactly zero (the
    fluxes are formed exactly in integer fixed point, so the cancelling
    terms are equal)."""
    c = np.full((10, 9, 12), 2.5)
    t = inputs.tzc(8, 3)
    su, sv, sw = run_advect(c, c, c, t, t)
    for s in (su, sv, sw):
        assert np.all(s[1:-1, 1:-1, 1:-1] == 0.0)


@pytest.mark.parametrize("scale", [1e150, 1e-150, -3.0])
def test_advect_extreme_magnitudes(scale):
    """The fixed-point scale follows the fields' magnitude (here 10^150 and
    10^-150 times the benchmark winds, and a negated copy)."""
    u, v, w = (scale * a for a in inputs.winds(40, 24, 10, seeds=(11, 12, 13)))
    t1, t2 = inputs.tzc(10, 7), inputs.tzc(10, 8)
    ref = oracle.advect_uvw(u, v, w, t1, t2, 0.25, 0.25)
    got = run_advect(u, v, w, t1, t2)
    for g, r in zip(got, ref):
        assert rel_err(g, r) <= 1e-13


@pytest.mark.parametrize("case", ["small_w", "small_tcy", "zero_v"])
def test_advect_uneven_magnitudes(case):
    """Fields or factors whose magnitudes differ by more than 2^8 are
    evaluated in binary64 (a single fixed-point scale would cost the small
    one its precision); a field that is identically zero keeps the
    fixed-point path.  Either way the result matches the oracle."""
    u, v, w = inputs.winds(33, 20, 9, seeds=(21, 22, 23))
    t1, t2 = inputs.tzc(9, 7), inputs.tzc(9, 8)
    tcy = 0.25
    if case == "small_w":
        w = w * 1e-7
    elif case == "small_tcy":
        tcy = 0.25e-6
    else:
        v = np.zeros_like(v)
    ref = oracle.advect_uvw(u, v, w, t1, t2, 0.25, tcy)
    got = run_advect(u, v, w, t1, t2, tcy=tcy)
    for g, r in zip(got, ref):
        assert rel_err(g, r) <= 1e-13
    # the binary64 path rounds every operation in the oracle's order
    if case != "zero_v":
        for g, r in zip(got, ref):
            assert np.array_equal(g, r)


def test_advect_nonfinite_propagates():
    """A NaN in u: the launch falls back to binary64, so exactly the cells
    whose stencil reads it are NaN, as in the oracle, and the rest match."""
    u, v, w = inputs.winds(20, 16, 8, seeds=(31, 32, 33))
    u[4, 5, 6] = np.nan
    t1, t2 = inputs.tzc(8, 7), inputs.tzc(8, 8)
    ref = oracle.advect_uvw(u, v, w, t1, t2, 0.25, 0.25)
    got = run_advect(u, v, w, t1, t2)
    inner = (slice(1, -1),) * 3
    for g, r in zip(got, ref):
        g, r = g[inner], r[inner]
        assert np.array_equal(np.isnan(g), np.isnan(r)) and np.isnan(r).any()
        ok = ~np.isnan(r)
        assert np.max(np.abs(g[ok] - r[ok])) <= 1e-13 * np.max(np.abs(r[ok]))
