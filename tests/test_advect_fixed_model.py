"""Host model of the advection kernel's integer arithmetic.

The kernel (stencil_advect_uvw's fixed-point path) quantises u, v, w as
X = trunc(x 2^S), forms each flux product a (b + c) from three 32 x 32-bit
partial products, takes the self terms um (u + um) - up (u + up) as the one
product (um - up)(u + um + up), multiplies by the quantised factors the
same way (a shift for power-of-two tcx, tcy) and rounds each tendency once.
This file restates that arithmetic with Python integers, checks every
product's error bound exactly, and compares the model with the oracle on
small fields: the readings the kernel relies on (the factored self term,
the truncated products) stay within 1e-13 of the written formula, and
constant fields still give exactly zero."""
import struct

import numpy as np
import pytest

import oracle
from paper_2310_01882_b300 import inputs


def _bits(x):
    return struct.unpack("<Q", struct.pack("<d", float(x)))[0]


def _s32(x):
    x &= (1 << 32) - 1
    return x - (1 << 32) if x >> 31 else x


def _ceil_log2_bits(b):
    e = (b >> 52) - 1023
    return e + 1 if (b & ((1 << 52) - 1)) else e


def _trunc(x, S):
    """trunc(x 2^S) toward zero, from the significand (the kernel's fx_trunc)."""
    b = _bits(x)
    e = (b >> 52) & 0x7FF
    m = ((b & ((1 << 52) - 1)) | (1 << 52)) << 10
    q = m >> min(1085 - e - S, 63)
    return -q if b >> 63 else q


def _round(x, S):
    """round(x 2^S), halves away from zero (the factors' quantiser)."""
    b = _bits(x)
    e = (b >> 52) & 0x7FF
    if e == 0:
        return 0
    m = (b & ((1 << 52) - 1)) | (1 << 52)
    sh = e - 1075 + S
    q = m << sh if sh >= 0 else ((m + (1 << (-sh - 1))) >> -sh if sh > -64 else 0)
    return -q if b >> 63 else q


def mh(a, s):
    """a s / 2^64 from three signed 32 x 32-bit products; asserts the
    operand ranges and that the result is within [-1/4, 9/4) of exact."""
    assert abs(a) <= 2 ** 62 and abs(s) < 2 ** 63 - 2 ** 32
    al, sl = _s32(a), _s32(s)
    ah = _s32(a >> 32) + ((a & 0xFFFFFFFF) >> 31)
    sh = _s32(s >> 32) + ((s & 0xFFFFFFFF) >> 31)
    assert ah * 2 ** 32 + al == a and sh * 2 ** 32 + sl == s
    t = ((ah * sl) >> 32) + ((al * sh) >> 32)
    assert -(2 ** 31) <= t < 2 ** 31
    r = ah * sh + t
    d = a * s - r * 2 ** 64  # exact
    assert -(2 ** 62) <= d < 9 * 2 ** 62
    return r


def model(u, v, w, t1, t2, tcx, tcy):
    nz2, ny2, nx2 = u.shape
    M = max(_bits(np.max(np.abs(a))) for a in (u, v, w))
    cmax = max(_bits(abs(c)) for c in [tcx, tcy, *t1, *t2])
    S = 61 - _ceil_log2_bits(M)
    T = 62 - _ceil_log2_bits(cmax)
    Q = 2 * S + T - 128
    U, V, W = ([[[_trunc(a[k, j, i], S) for i in range(nx2)] for j in range(ny2)] for k in range(nz2)]
               for a in (u, v, w))
    cx, cy = _round(tcx, T), _round(tcy, T)
    pow2 = cx > 0 and cy > 0 and (cx & (cx - 1)) == 0 and (cy & (cy - 1)) == 0

    def hf(c, d):
        if pow2:
            sh = 64 - (c.bit_length() - 1)
            assert 1 <= sh <= 31
            return d >> sh
        return mh(c, d)

    out = [np.zeros_like(u) for _ in range(3)]
    for k in range(1, nz2 - 1):
        c1, c2 = _round(t1[k - 1], T), _round(t2[k - 1], T)
        for j in range(1, ny2 - 1):
            for i in range(1, nx2 - 1):
                def g(A, di=0, dj=0, dk=0):
                    return A[k + dk][j + dj][i + di]
                u0, v0, w0 = g(U), g(V), g(W)
                um, up, vm, vp, wm, wp = g(U, -1), g(U, 1), g(V, 0, -1), g(V, 0, 1), g(W, 0, 0, -1), g(W, 0, 0, 1)
                terms = [
                    (mh(um - up, u0 + um + up),
                     mh(g(U, 0, -1), g(V, 0, -1) + g(V, 1, -1)) - mh(g(U, 0, 1), v0 + g(V, 1)),
                     mh(g(U, 0, 0, -1), wm + g(W, 1, 0, -1)), mh(g(U, 0, 0, 1), w0 + g(W, 1))),
                    (mh(g(V, -1), g(U, -1) + g(U, -1, 1)) - mh(g(V, 1), u0 + g(U, 0, 1)),
                     mh(vm - vp, v0 + vm + vp),
                     mh(g(V, 0, 0, -1), wm + g(W, 0, 1, -1)), mh(g(V, 0, 0, 1), w0 + g(W, 0, 1))),
                    (mh(g(W, -1), g(U, -1) + g(U, -1, 0, 1)) - mh(g(W, 1), u0 + g(U, 0, 0, 1)),
                     mh(g(W, 0, -1), vm + g(V, 0, -1, 1)) - mh(g(W, 0, 1), v0 + g(V, 0, 0, 1)),
                     mh(wm, w0 + wm), mh(wp, w0 + wp)),
                ]
                for o, (dx, dy, p3, p4) in zip(out, terms):
                    s = hf(cx, dx) + hf(cy, dy) + mh(c1, p3) - mh(c2, p4)
                    assert abs(s) < 2 ** 63
                    o[k, j, i] = float(s) * 2.0 ** (-Q)  # one rounding (the kernel: convert, scale exactly)
    return out


def _rel(g, r):
    inner = (slice(1, -1),) * 3
    return np.max(np.abs(g[inner] - r[inner])) / np.max(np.abs(r[inner]))


@pytest.mark.parametrize("nx,ny,nz,scale,tcy", [(9, 7, 5, 1.0, 0.25), (8, 6, 4, 1e150, 0.25),
                                                (7, 5, 4, -3e-150, 0.25), (7, 6, 5, 1.0, 0.3)])
def test_model_matches_oracle(nx, ny, nz, scale, tcy):
    u, v, w = (scale * a for a in inputs.winds(nx, ny, nz, seeds=(4, 5, 6)))
    t1, t2 = inputs.tzc(nz, 7), inputs.tzc(nz, 8)
    ref = oracle.advect_uvw(u, v, w, t1, t2, 0.25, tcy)
    for g, r in zip(model(u, v, w, t1, t2, 0.25, tcy), ref):
        assert _rel(g, r) <= 1e-14


def test_model_constant_fields_exact_zero():
    c = np.full((6, 7, 8), 2.5)
    t = inputs.tzc(4, 3)
    for s in model(c, c, c, t, t, 0.25, 0.25):
        assert np.all(s == 0.0)


def test_truncation_is_odd_and_within_one_unit():
    from fractions import Fraction
    rng = np.random.default_rng(3)
    for x in list(rng.standard_normal(200) * 7.0) + [0.0, 5e-324, -2.0 ** -40]:
        q = _trunc(float(x), 58)
        assert q == -_trunc(-float(x), 58)
        exact = Fraction(float(x)) * 2 ** 58
        assert abs(exact - q) < 1 and (q == 0 or (q > 0) == (exact > 0))
