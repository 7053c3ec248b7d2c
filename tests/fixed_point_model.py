"""A CPU model of the integer arithmetic of the library's FP64 fixed-point
Jacobi sweep (the resident form: the iterate held as integers for the whole
call), in exact integer numpy arithmetic.  Test infrastructure: it documents
what the kernel computes, lets the host tests show why the scale rule
matters, and a GPU test checks that the kernel's results equal the model's
bit for bit.  It is not the oracle (the oracle is the binary64 definition,
oracle/).

Values are integers q at a scale S (x = q * 2^-S).  One sweep of the
interior is q' = floor((q[i-1] + q[i+1] + q[j-1] + q[j+1] + q[k-1] + q[k+1]
+ g + 3) / 6), the sum exact, i.e. the average rounded to the nearest unit
(halves up), with g the source h*h*f at the same scale.

Two rules for S:
  * `call_scale` (the rule of earlier builds): one S for the whole call from
    an a-priori bound on every iterate,
    M = min(max|u| + n h^2 max|f| / 6, 3 max|u| + max|f| L^2 / 4),
    S = 58 - ceil(log2(6 M + h^2 max|f|)); conversions of negative values
    truncated toward zero.
  * `pass_scale` (the kernel's rule): every pass computes at the scale its
    input is stored at and writes its output at a scale chosen from a bound
    on what it produces (the largest magnitude the previous pass wrote, the
    Dirichlet values and the source's contribution over the pass); the scale
    changes only when it must grow coarser or can grow at least two steps
    finer, and a pass that changes it shifts the values it writes.  The
    source enters every pass converted at the computing scale from
    binary64; conversions round halves away from zero.
"""
import math

import numpy as np

I3 = (slice(1, -1),) * 3


def _exp(x):
    """frexp exponent: x = m 2^e with m in [0.5, 1) (0 for x = 0)."""
    return math.frexp(x)[1] if x > 0 else 0


def scale_for(B):
    return min(58 - _exp(B), 1022)


def _round_half_away(y):
    """y: float64 array holding exact multiples of a power of two (an ldexp
    of binary64 values); round to nearest integer, halves away from zero."""
    a = np.abs(y)
    fl = np.floor(a)
    r = fl + (a - fl >= 0.5)
    return np.where(y < 0, -r, r).astype(np.int64)


def quantise(x, S, truncate_negatives=False):
    y = np.ldexp(np.asarray(x, dtype=np.float64), S)  # exact while |y| < 2^1023
    if truncate_negatives:
        a = np.abs(y)
        fl = np.floor(a)
        r = np.where(y < 0, fl, fl + (a - fl >= 0.5))
        return np.where(y < 0, -r, r).astype(np.int64)
    return _round_half_away(y)


def quantise_source(f, hh, S, truncate_negatives=False):
    """round(f * hh * 2^S) of the exact product (not the rounded binary64
    product), as the kernel's 64x64-bit multiply of significands gives."""
    mh, eh = math.frexp(hh)
    Mh = int(mh * 2 ** 53)
    flat = np.asarray(f, dtype=np.float64).ravel()
    out = np.empty(flat.size, dtype=np.int64)
    for idx, v in enumerate(flat.tolist()):
        if v == 0.0:
            out[idx] = 0
            continue
        mf, ef = math.frexp(abs(v))
        Mf = int(mf * 2 ** 53)
        num = Mf * Mh                       # |f hh| = num * 2^(ef + eh - 106)
        sh = ef + eh - 106 + S              # |f hh| 2^S = num * 2^sh
        if sh >= 0:
            r = num << sh
        else:
            t = num >> (-sh - 1)            # floor(2 |x| 2^S)
            r = t >> 1 if truncate_negatives and v < 0 else (t + 1) >> 1
        out[idx] = -r if v < 0 else r
    return out.reshape(np.shape(f))


def _sweep(Q, g):
    s = Q[1:-1, 1:-1, :-2] + Q[1:-1, 1:-1, 2:]
    s = s + Q[1:-1, :-2, 1:-1]
    s = s + Q[1:-1, 2:, 1:-1]
    s = s + Q[:-2, 1:-1, 1:-1]
    s = s + Q[2:, 1:-1, 1:-1]
    s = s + g
    out = Q.copy()
    out[I3] = (s + 3) // 6
    return out


def _halo_mask(shape):
    m = np.ones(shape, dtype=bool)
    m[I3] = False
    return m


def call_scale(u0, f, h, nsweeps):
    """nsweeps sweeps with one a-priori scale for the call (earlier rule)."""
    hh = h * h
    nz, ny, nx = (s - 2 for s in u0.shape)
    maxu = float(np.max(np.abs(u0)))
    maxf = float(np.max(np.abs(f[I3])))
    lmin = (min(nx, ny, nz) + 1) * h
    M = min(maxu + nsweeps * hh * maxf / 6.0, 3.0 * maxu + maxf * lmin * lmin / 4.0)
    S = scale_for(6.0 * M + hh * maxf)
    Q = quantise(u0, S, truncate_negatives=True)
    G = quantise_source(f[I3], hh, S, truncate_negatives=True)
    for _ in range(nsweeps):
        Q = _sweep(Q, G)
    out = np.array(u0, dtype=np.float64, copy=True)
    out[I3] = np.ldexp(Q[I3].astype(np.float64), -S)
    return out


def pass_scale(u0, f, h, nsweeps, T=1, trace=None):
    """nsweeps sweeps, T per pass, with the per-pass scale rule.  `trace`
    (a list) receives the scale each pass writes its output at."""
    hh = h * h
    halo = _halo_mask(u0.shape)
    mh = float(np.max(np.abs(u0[halo])))
    mu = float(np.max(np.abs(u0[I3])))
    maxf = float(np.max(np.abs(f[I3])))
    hmf = hh * maxf
    T1 = min(T, nsweeps)
    S = scale_for(6.0 * (max(mu, mh) + T1 * hmf / 6.0) + hmf)   # set-up: slot 0
    key = int(math.ldexp(mu, S - 32))
    Q = quantise(u0, S)
    G, GS = quantise_source(f[I3], hh, S), S
    left = nsweeps
    while left > 0:
        t = min(T, left)
        # the scale this pass writes at, from the bound on what it produces
        Mi = math.ldexp(key + 1.0, 32 - S)
        M = max(Mi, mh) + t * hmf / 6.0
        So = scale_for(6.0 * M + hmf)
        if S <= So < S + 2:
            So = S
        # compute at the stored scale S (the source converted at S)
        q = Q[I3]
        Q = quantise(np.where(halo, u0, 0.0), S)   # Dirichlet values at the computing scale
        Q[I3] = q
        if GS != S:
            G, GS = quantise_source(f[I3], hh, S), S
        for _ in range(t):
            Q = _sweep(Q, G)
        d = max(-62, min(62, So - S))
        q = Q[I3]
        if d > 0:
            q = q << d
        elif d < 0:
            q = (q + (1 << (-d - 1))) >> (-d)
        Q[I3] = q
        S = So
        key = int(np.max(np.abs(q >> 32)))
        if trace is not None:
            trace.append(S)
        left -= t
    out = np.array(u0, dtype=np.float64, copy=True)
    out[I3] = np.ldexp(Q[I3].astype(np.float64), -S)
    return out
