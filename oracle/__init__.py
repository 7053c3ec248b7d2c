"""CPU oracle for the stencil hot path -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
import this package.  The product library (paper_2310_01882_b300) never
imports it and shares no code with it.

Fields are numpy arrays of shape (nz+2, ny+2, nx+2) (x fastest, one-cell
halo), float64 unless stated.  The arithmetic lives in oracle.c (plain C
loops); this module only marshals arrays.  exact.py holds the closed-form
discrete Poisson solution used as a pin.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        # ORACLE_LIB points the pins at a deliberately broken build (the
        # mutation test); normally the library is built from oracle.c.
        path = os.environ.get("ORACLE_LIB") or _build.build()
        L = ctypes.CDLL(path)
        d, i64, i32, p = ctypes.c_double, ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
        f32 = ctypes.c_float
        L.oracle_jacobi_sweep_f64.argtypes = [p, p, p, i64, i64, i64, d, i32]
        L.oracle_jacobi_f64.argtypes = [p, p, p, i64, i64, i64, d, i64, i32]
        L.oracle_jacobi_sweep_f32.argtypes = [p, p, p, i64, i64, i64, f32]
        L.oracle_jacobi_sweep_bf16.argtypes = [p, p, p, i64, i64, i64, f32]
        L.oracle_f32_to_bf16.argtypes = [p, p, i64]
        L.oracle_bf16_to_f32.argtypes = [p, p, i64]
        L.oracle_residual_f64.argtypes = [p, p, i64, i64, i64, d, p, p, i32]
        L.oracle_rbgs_f64.argtypes = [p, p, i64, i64, i64, d, i64, i32]
        L.oracle_average2d.argtypes = [p, p, i64, i64, i64, i64]
        L.oracle_apply_linear.argtypes = [p, p, i64, i64, i64, p, p, i32]
        L.oracle_rbgs_f32.argtypes = [p, p, i64, i64, i64, f32, i64]
        L.oracle_rbgs_bf16.argtypes = [p, p, i64, i64, i64, f32, i64]
        L.oracle_advect_uvw.argtypes = [p, p, p, p, p, p, p, p, d, d, i64, i64, i64, i32]
        L.oracle_refine.argtypes = [p, p, i64, i64, i64, d, d, i32, i32, i64, i64, d, p, p, i64, p, p, p]
        L.oracle_refine.restype = i64
        L.oracle_num_threads.argtypes = [i32]
        L.oracle_num_threads.restype = i32
        _lib = L
    return _lib


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def _dims(a):
    nz2, ny2, nx2 = a.shape
    return nx2 - 2, ny2 - 2, nz2 - 2


def _c64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def num_threads(nthreads=0):
    return lib().oracle_num_threads(nthreads)


def jacobi_sweep(u, f, h, nthreads=1):
    """One FP64 Jacobi sweep; returns a new field (halo copied from u)."""
    u, f = _c64(u), _c64(f)
    out = np.empty_like(u)
    nx, ny, nz = _dims(u)
    lib().oracle_jacobi_sweep_f64(_ptr(u), _ptr(out), _ptr(f), nx, ny, nz, h, nthreads)
    return out


def jacobi(u, f, h, nsweeps, nthreads=1):
    """nsweeps FP64 Jacobi sweeps; returns a new field."""
    u = np.array(u, dtype=np.float64, order="C", copy=True)
    f = _c64(f)
    tmp = np.empty_like(u)
    nx, ny, nz = _dims(u)
    lib().oracle_jacobi_f64(_ptr(u), _ptr(tmp), _ptr(f), nx, ny, nz, h, nsweeps, nthreads)
    return u


def jacobi_run(u, tmp, f, h, nsweeps, nthreads=1):
    """nsweeps FP64 Jacobi sweeps on caller-owned C-contiguous float64
    buffers: the result ends in u, tmp is scratch (the timed CPU baselines
    reuse their buffers across calls)."""
    assert u.dtype == np.float64 and u.flags.c_contiguous and tmp.shape == u.shape and f.shape == u.shape
    assert tmp.dtype == np.float64 and tmp.flags.c_contiguous and f.dtype == np.float64 and f.flags.c_contiguous
    nx, ny, nz = _dims(u)
    lib().oracle_jacobi_f64(_ptr(u), _ptr(tmp), _ptr(f), nx, ny, nz, h, nsweeps, nthreads)
    return u


def f32_coeff(h):
    """The FP32 coefficient h*h used by FP32-arithmetic sweeps (rounded once)."""
    return np.float32(np.float64(h) * np.float64(h))


def jacobi_sweep_f32(u, f, h):
    """One sweep with FP32 storage and FP32 arithmetic (inputs float32)."""
    u = np.ascontiguousarray(u, dtype=np.float32)
    f = np.ascontiguousarray(f, dtype=np.float32)
    out = np.empty_like(u)
    nx, ny, nz = _dims(u)
    lib().oracle_jacobi_sweep_f32(_ptr(u), _ptr(out), _ptr(f), nx, ny, nz, f32_coeff(h))
    return out


def to_bf16(a):
    """Round float32 values to bf16 (RNE); returns uint16 bit patterns."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    out = np.empty(a.shape, dtype=np.uint16)
    lib().oracle_f32_to_bf16(_ptr(a), _ptr(out), a.size)
    return out


def from_bf16(b):
    """bf16 bit patterns (uint16) to float32."""
    b = np.ascontiguousarray(b, dtype=np.uint16)
    out = np.empty(b.shape, dtype=np.float32)
    lib().oracle_bf16_to_f32(_ptr(b), _ptr(out), b.size)
    return out


def jacobi_sweep_bf16(u16, f16, h):
    """One sweep with bf16 storage (uint16 bit patterns), FP32 arithmetic."""
    u16 = np.ascontiguousarray(u16, dtype=np.uint16)
    f16 = np.ascontiguousarray(f16, dtype=np.uint16)
    out = np.empty_like(u16)
    nx, ny, nz = _dims(u16)
    lib().oracle_jacobi_sweep_bf16(_ptr(u16), _ptr(out), _ptr(f16), nx, ny, nz, f32_coeff(h))
    return out


def average2d(u, nsweeps):
    """nsweeps sweeps of the 2D four-neighbour average on every z plane;
    returns a new field."""
    u = np.array(u, dtype=np.float64, order="C", copy=True)
    tmp = np.empty_like(u)
    nx, ny, nz = _dims(u)
    lib().oracle_average2d(_ptr(u), _ptr(tmp), nx, ny, nz, nsweeps)
    return u


def apply_linear(u, offsets, coeffs, out=None):
    """out(x) = sum_p coeffs[p] * u(x + offsets[p]) on the interior points
    whose reads lie in the field (offsets: (npoints, 3) ints dx, dy, dz in
    [-3, 3]; with r = max |d|, indices r .. n + 1 - r); the rest of out is
    out's own (zeros if out is None)."""
    u = _c64(u)
    out = np.zeros_like(u) if out is None else np.array(out, dtype=np.float64, order="C", copy=True)
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32).reshape(-1, 3))
    c = _c64(np.asarray(coeffs, dtype=np.float64).reshape(-1))
    assert off.shape[0] == c.size and np.all(np.abs(off) <= 3)
    nx, ny, nz = _dims(u)
    lib().oracle_apply_linear(_ptr(u), _ptr(out), nx, ny, nz, _ptr(off), _ptr(c), c.size)
    return out


def rbgs(u, f, h, nsweeps, nthreads=1):
    """nsweeps red-black Gauss-Seidel sweeps in FP64; returns a new field."""
    u = np.array(u, dtype=np.float64, order="C", copy=True)
    f = _c64(f)
    nx, ny, nz = _dims(u)
    lib().oracle_rbgs_f64(_ptr(u), _ptr(f), nx, ny, nz, h, nsweeps, nthreads)
    return u


def rbgs_f32(u, f, h, nsweeps):
    """Red-black sweeps with FP32 storage and arithmetic (inputs float32)."""
    u = np.array(u, dtype=np.float32, order="C", copy=True)
    f = np.ascontiguousarray(f, dtype=np.float32)
    nx, ny, nz = _dims(u)
    lib().oracle_rbgs_f32(_ptr(u), _ptr(f), nx, ny, nz, f32_coeff(h), nsweeps)
    return u


def rbgs_bf16(u16, f16, h, nsweeps):
    """Red-black sweeps with bf16 storage (uint16 bit patterns), FP32 arithmetic."""
    u16 = np.array(u16, dtype=np.uint16, order="C", copy=True)
    f16 = np.ascontiguousarray(f16, dtype=np.uint16)
    nx, ny, nz = _dims(u16)
    lib().oracle_rbgs_bf16(_ptr(u16), _ptr(f16), nx, ny, nz, f32_coeff(h), nsweeps)
    return u16


def residual(u, f, h, want_r=False, nthreads=1):
    """FP64 residual r = f - A u.  Returns (norm_r, norm_f[, r])."""
    u, f = _c64(u), _c64(f)
    nx, ny, nz = _dims(u)
    norms = np.zeros(2, dtype=np.float64)
    r = np.zeros_like(u) if want_r else None
    lib().oracle_residual_f64(_ptr(u), _ptr(f), nx, ny, nz, h,
                              _ptr(r) if want_r else None, _ptr(norms), nthreads)
    if want_r:
        return norms[0], norms[1], r
    return norms[0], norms[1]


def advect_uvw(u, v, w, tzc1, tzc2, tcx, tcy, nthreads=1):
    """PW advection tendencies (su, sv, sw); interior written, halo zero."""
    u, v, w = _c64(u), _c64(v), _c64(w)
    tzc1, tzc2 = _c64(tzc1), _c64(tzc2)
    nx, ny, nz = _dims(u)
    assert tzc1.shape == (nz,) and tzc2.shape == (nz,)
    su, sv, sw = (np.zeros_like(u) for _ in range(3))
    lib().oracle_advect_uvw(_ptr(u), _ptr(v), _ptr(w), _ptr(su), _ptr(sv), _ptr(sw),
                            _ptr(tzc1), _ptr(tzc2), tcx, tcy, nx, ny, nz, nthreads)
    return su, sv, sw


INNER_CODES = {"f64": 0, "f32": 1, "bf16": 2}


def refine(u0, f, h, rtol, inner="f32", m=100, max_sweeps=10 ** 7, stall_ratio=0.9999, smoother="jacobi"):
    """Mixed-precision refinement (see oracle_refine; smoother "jacobi" or
    "redblack" for the inner sweeps).  Returns a dict with
    u, sweeps, cycles, hist (rel of each residual evaluated), rel (final),
    final_inner and status (0 converged, -7 not converged / stalled,
    -6 non-finite)."""
    u = np.array(u0, dtype=np.float64, order="C", copy=True)
    f = _c64(f)
    nx, ny, nz = _dims(u)
    hist_len = 100000
    hist = np.zeros(hist_len, dtype=np.float64)
    cycles = np.zeros(1, dtype=np.int64)
    fin = np.zeros(1, dtype=np.int32)
    status = np.zeros(1, dtype=np.int32)
    work = np.zeros(6 * u.size, dtype=np.float64)
    sweeps = lib().oracle_refine(_ptr(u), _ptr(f), nx, ny, nz, h, rtol, INNER_CODES[inner],
                                 {"jacobi": 0, "redblack": 1}[smoother], m,
                                 max_sweeps, stall_ratio, _ptr(cycles), _ptr(hist), hist_len,
                                 _ptr(fin), _ptr(status), _ptr(work))
    c = int(cycles[0])
    inv = {v: k for k, v in INNER_CODES.items()}
    n_hist = min(c + 1, hist_len)
    return {"u": u, "sweeps": int(sweeps), "cycles": c, "hist": hist[:n_hist].copy(),
            "final_inner": inv[int(fin[0])], "rel": float(hist[n_hist - 1]), "status": int(status[0])}
