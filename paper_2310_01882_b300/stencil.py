"""Thin Python binding of libstencil.so (include/stencil.h).

Argument marshalling only: every step of the computation runs in the CUDA
library.  Fields live in torch CUDA tensors (torch is used for device memory
and streams); the binding passes their raw device pointers and strides
across the C ABI.  If the library has not been built, the first call raises;
there is no fallback.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libstencil.so")

F64, F32, BF16 = 0, 1, 2
SWEEP_AUTO, SWEEP_FP64_NATIVE, SWEEP_FP64_FIXED = 0, 1, 2

OK = 0
ERRORS = {
    -1: "STENCIL_ERR_ARG", -2: "STENCIL_ERR_ALIGN", -3: "STENCIL_ERR_DTYPE", -4: "STENCIL_ERR_CUDA",
    -5: "STENCIL_ERR_TIMEOUT", -6: "STENCIL_ERR_NONFINITE", -7: "STENCIL_ERR_NOT_CONVERGED",
    -8: "STENCIL_ERR_RANGE",
}
ELEM = {F64: 8, F32: 4, BF16: 2}


class StencilError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class stencil_grid(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("nx", ctypes.c_int64), ("ny", ctypes.c_int64),
                ("nz", ctypes.c_int64), ("sy", ctypes.c_int64), ("sz", ctypes.c_int64),
                ("dtype", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class stencil_problem(ctypes.Structure):
    _fields_ = [("u", stencil_grid), ("f", stencil_grid), ("h", ctypes.c_double)]


class stencil_batch_opts(ctypes.Structure):
    _fields_ = [("rtol", ctypes.c_double), ("max_sweeps", ctypes.c_int64), ("inner_dtype", ctypes.c_int32),
                ("sweeps_per_cycle", ctypes.c_int32), ("sweeps_per_pass", ctypes.c_int32),
                ("smoother", ctypes.c_int32), ("stall_ratio", ctypes.c_double)]


class stencil_result(ctypes.Structure):
    _fields_ = [("sweeps", ctypes.c_int64), ("cycles", ctypes.c_int32), ("status", ctypes.c_int32),
                ("rel_residual", ctypes.c_double), ("final_dtype", ctypes.c_int32), ("reserved", ctypes.c_int32)]


_lib = None

# Every exported symbol of include/stencil.h, with its ctypes signature.
_P = ctypes.c_void_p
_G = ctypes.POINTER(stencil_grid)
SIGNATURES = {
    "stencil_version": ([], ctypes.c_char_p),
    "stencil_last_error": ([], ctypes.c_char_p),
    "stencil_ctx_create": ([ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "stencil_ctx_destroy": ([_P], ctypes.c_int),
    "stencil_ctx_status": ([_P, _P], ctypes.c_int),
    "stencil_jacobi_sweep": ([_P, _G, _G, _G, _G, ctypes.c_double, ctypes.c_int64, ctypes.c_int32,
                              ctypes.c_int32, _P], ctypes.c_int),
    "stencil_average2d": ([_P, _G, _G, ctypes.c_int64, _P], ctypes.c_int),
    "stencil_apply_linear": ([_P, _G, _G, _P, _P, ctypes.c_int32, _P], ctypes.c_int),
    "stencil_apply_expr": ([_P, ctypes.POINTER(_G), ctypes.c_int32, _G, ctypes.c_char_p, _P], ctypes.c_int),
    "stencil_expr_source": ([ctypes.c_char_p, ctypes.c_int32, ctypes.c_char_p, ctypes.c_size_t,
                             ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
    "stencil_redblack_sweep": ([_P, _G, _G, _G, _G, ctypes.c_double, ctypes.c_int64, ctypes.c_int32,
                                ctypes.c_int32, _P], ctypes.c_int),
    "stencil_residual": ([_P, _G, _G, ctypes.c_double, _G, _P, _P], ctypes.c_int),
    "stencil_advect_uvw": ([_P, _G, _G, _G, _G, _G, _G, _P, _P, ctypes.c_double, ctypes.c_double, _P],
                           ctypes.c_int),
    "stencil_residual_noalloc": ([_G, _G, ctypes.c_double, _G, _P, _P], ctypes.c_int),
    "stencil_autotune_sweep": ([_P, _G, _G, _G, _G, ctypes.c_double, ctypes.c_int32, ctypes.c_char_p, ctypes.c_size_t,
                                _P], ctypes.c_int),
    "stencil_sweep_config_count": ([ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                    ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
    "stencil_sweep_config_select": ([_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                     ctypes.c_int32], ctypes.c_int),
    "stencil_redblack_config_count": ([ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                       ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
    "stencil_redblack_config_select": ([_P, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                        ctypes.c_int32], ctypes.c_int),
    "stencil_residual_config_count": ([ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
    "stencil_residual_config_select": ([_P, ctypes.c_int32], ctypes.c_int),
    "stencil_advect_config_count": ([ctypes.POINTER(ctypes.c_int32)], ctypes.c_int),
    "stencil_advect_config_select": ([_P, ctypes.c_int32], ctypes.c_int),
    "wsnet_create": ([ctypes.c_int, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32), ctypes.c_int32,
                      ctypes.c_uint64, ctypes.POINTER(ctypes.c_void_p)], ctypes.c_int),
    "wsnet_destroy": ([_P], ctypes.c_int),
    "wsnet_num_params": ([_P, ctypes.POINTER(ctypes.c_int64)], ctypes.c_int),
    "wsnet_get_params": ([_P, _P, ctypes.c_int64], ctypes.c_int),
    "wsnet_set_params": ([_P, _P, ctypes.c_int64], ctypes.c_int),
    "wsnet_infer": ([_P, _G, _G, _P], ctypes.c_int),
    "wsnet_train_step": ([_P, _G, _G, ctypes.c_int32, ctypes.c_float, ctypes.POINTER(ctypes.c_double), _P],
                         ctypes.c_int),
    "wsnet_use_tcgen05": ([_P, ctypes.c_int32], ctypes.c_int),
    "wsnet_save": ([_P, ctypes.c_char_p], ctypes.c_int),
    "wsnet_load": ([_P, ctypes.c_char_p], ctypes.c_int),
    "wsnet_status": ([_P, _P], ctypes.c_int),
    "wsnet_loss_grad": ([_P, _P, _P, _P, _P, ctypes.POINTER(ctypes.c_double), _P], ctypes.c_int),
    "stencil_batch_workspace_size": ([ctypes.POINTER(stencil_problem), ctypes.c_int32,
                                      ctypes.POINTER(ctypes.c_size_t)], ctypes.c_int),
    "stencil_batch_solve": ([_P, ctypes.POINTER(stencil_problem), ctypes.c_int32,
                             ctypes.POINTER(stencil_batch_opts), _P, ctypes.c_size_t,
                             ctypes.POINTER(stencil_result), _P], ctypes.c_int),
}


def lib():
    """Load libstencil.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2310_01882_b300.build`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (args, res) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def _check(rc):
    if rc != OK:
        raise StencilError(rc, lib().stencil_last_error().decode())
    return rc


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Field:
    """A halo-padded 3D field in a torch CUDA tensor.

    Storage shape (nz+2, ny+2, sy) with sy = nx+2 rounded up to 16 bytes, so
    every row starts 16-byte aligned; `.cells` is the (nz+2, ny+2, nx+2)
    view of the grid cells, halo included (x fastest)."""

    TORCH_DTYPES = None

    def __init__(self, nx, ny, nz, dtype=F64, device="cuda", storage=None):
        import torch
        if Field.TORCH_DTYPES is None:
            Field.TORCH_DTYPES = {F64: torch.float64, F32: torch.float32, BF16: torch.bfloat16}
        self.nx, self.ny, self.nz, self.dtype = int(nx), int(ny), int(nz), dtype
        g = 16 // ELEM[dtype]
        self.sy = (self.nx + 2 + g - 1) // g * g
        if storage is None:
            storage = torch.zeros((self.nz + 2, self.ny + 2, self.sy), dtype=Field.TORCH_DTYPES[dtype],
                                  device=device)
        assert storage.shape == (self.nz + 2, self.ny + 2, self.sy) and storage.is_contiguous()
        self.storage = storage
        self.sz = self.sy * (self.ny + 2)

    @property
    def cells(self):
        return self.storage[:, :, : self.nx + 2]

    def grid(self):
        return stencil_grid(self.storage.data_ptr(), self.nx, self.ny, self.nz, self.sy, self.sz,
                            self.dtype, 0)

    @classmethod
    def from_numpy(cls, a, dtype=F64, device="cuda"):
        """a: (nz+2, ny+2, nx+2) array (float64/float32; bf16 is rounded RNE)."""
        import torch
        nz, ny, nx = (s - 2 for s in a.shape)
        f = cls(nx, ny, nz, dtype, device)
        src = torch.from_numpy(np.ascontiguousarray(a))
        f.cells.copy_(src.to(device=device, dtype=Field.TORCH_DTYPES[dtype]))
        return f

    def to_numpy(self, dtype=np.float64):
        import torch
        return self.cells.to(torch.float64).cpu().numpy().astype(dtype, copy=False)

    def like(self):
        return Field(self.nx, self.ny, self.nz, self.dtype, self.storage.device)


class Context:
    """Owns a stencil_ctx (its device scratch memory)."""

    def __init__(self, device=0):
        h = ctypes.c_void_p()
        _check(lib().stencil_ctx_create(int(device), ctypes.byref(h)))
        self.handle = h

    def close(self):
        if self.handle:
            lib().stencil_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def stencil_version():
    return lib().stencil_version().decode()


def stencil_ctx_status(ctx, stream=None):
    return _check(lib().stencil_ctx_status(ctx.handle, _stream(stream)))


def stencil_jacobi_sweep(ctx, u, u_tmp, f, work, h, nsweeps, sweeps_per_pass=0, flags=SWEEP_AUTO,
                         stream=None):
    """work: None or an F64 Field of u's extents (see include/stencil.h)."""
    gu, gt, gf = u.grid(), u_tmp.grid(), f.grid()
    gw = work.grid() if work is not None else None
    return _check(lib().stencil_jacobi_sweep(ctx.handle, ctypes.byref(gu), ctypes.byref(gt), ctypes.byref(gf),
                                             ctypes.byref(gw) if gw is not None else None,
                                             float(h), int(nsweeps), int(sweeps_per_pass), int(flags),
                                             _stream(stream)))


def stencil_apply_linear(ctx, inp, out, offsets, coeffs, stream=None):
    """out = sum_p coeffs[p] * inp(. + offsets[p]) on the interior points whose
    reads lie in the field (offsets: (npoints, 3) ints in -3..3; F64 Fields;
    see include/stencil.h)."""
    off = np.ascontiguousarray(np.asarray(offsets, dtype=np.int32).reshape(-1, 3))
    c = np.ascontiguousarray(np.asarray(coeffs, dtype=np.float64).reshape(-1))
    gi, go = inp.grid(), out.grid()
    return _check(lib().stencil_apply_linear(ctx.handle, ctypes.byref(gi), ctypes.byref(go),
                                             ctypes.c_void_p(off.ctypes.data), ctypes.c_void_p(c.ctypes.data),
                                             int(c.size) if c.size == off.shape[0] else -1, _stream(stream)))


def stencil_apply_expr(ctx, inputs, out, expr, stream=None):
    """out = expr over the F64 Fields `inputs` (a0, a1, ...) on the points
    whose reads lie in the field; the kernel is generated from expr and
    compiled at run time (see include/stencil.h for the grammar)."""
    grids = [f.grid() for f in inputs]
    arr = (_G * len(grids))(*[ctypes.pointer(g) for g in grids])
    go = out.grid()
    return _check(lib().stencil_apply_expr(ctx.handle, arr, len(grids), ctypes.byref(go), expr.encode(),
                                           _stream(stream)))


def stencil_expr_source(expr, ninputs):
    """(CUDA C source of the kernel stencil_apply_expr generates, radius)."""
    buf = ctypes.create_string_buffer(1 << 17)
    r = ctypes.c_int32(0)
    _check(lib().stencil_expr_source(expr.encode(), int(ninputs), buf, len(buf), ctypes.byref(r)))
    return buf.value.decode(), r.value


def stencil_average2d(ctx, u, u_tmp, nsweeps, stream=None):
    """The four-neighbour average on every z plane (F64 Fields)."""
    gu, gt = u.grid(), u_tmp.grid()
    return _check(lib().stencil_average2d(ctx.handle, ctypes.byref(gu), ctypes.byref(gt), int(nsweeps),
                                          _stream(stream)))


def stencil_redblack_sweep(ctx, u, u_tmp, f, work, h, nsweeps, sweeps_per_pass=0, flags=SWEEP_AUTO,
                           stream=None):
    """Red-black Gauss-Seidel sweeps; arguments as stencil_jacobi_sweep."""
    gu, gt, gf = u.grid(), u_tmp.grid(), f.grid()
    gw = work.grid() if work is not None else None
    return _check(lib().stencil_redblack_sweep(ctx.handle, ctypes.byref(gu), ctypes.byref(gt), ctypes.byref(gf),
                                               ctypes.byref(gw) if gw is not None else None,
                                               float(h), int(nsweeps), int(sweeps_per_pass), int(flags),
                                               _stream(stream)))


def stencil_autotune_sweep(ctx, u, u_tmp, f, work, h, flags=SWEEP_AUTO, stream=None):
    """Time every compiled sweep configuration on these grids and keep the
    fastest in ctx (see include/stencil.h).  Returns the text report."""
    gu, gt, gf = u.grid(), u_tmp.grid(), f.grid()
    gw = work.grid() if work is not None else None
    buf = ctypes.create_string_buffer(8192)
    _check(lib().stencil_autotune_sweep(ctx.handle, ctypes.byref(gu), ctypes.byref(gt), ctypes.byref(gf),
                                        ctypes.byref(gw) if gw is not None else None, float(h), int(flags),
                                        buf, len(buf), _stream(stream)))
    return buf.value.decode()


def stencil_sweep_config_count(dtype, flags, with_work, T):
    c = ctypes.c_int32()
    _check(lib().stencil_sweep_config_count(int(dtype), int(flags), int(bool(with_work)), int(T), ctypes.byref(c)))
    return c.value


def stencil_sweep_config_select(ctx, dtype, flags, with_work, T, index):
    return _check(lib().stencil_sweep_config_select(ctx.handle, int(dtype), int(flags), int(bool(with_work)),
                                                    int(T), int(index)))


def stencil_redblack_config_count(dtype, flags, with_work, sweeps_per_pass):
    c = ctypes.c_int32()
    _check(lib().stencil_redblack_config_count(int(dtype), int(flags), int(bool(with_work)), int(sweeps_per_pass),
                                               ctypes.byref(c)))
    return c.value


def stencil_redblack_config_select(ctx, dtype, flags, with_work, sweeps_per_pass, index):
    return _check(lib().stencil_redblack_config_select(ctx.handle, int(dtype), int(flags), int(bool(with_work)),
                                                       int(sweeps_per_pass), int(index)))


def stencil_residual_config_count():
    c = ctypes.c_int32()
    _check(lib().stencil_residual_config_count(ctypes.byref(c)))
    return c.value


def stencil_residual_config_select(ctx, index):
    return _check(lib().stencil_residual_config_select(ctx.handle, int(index)))


def stencil_advect_config_count():
    c = ctypes.c_int32(0)
    _check(lib().stencil_advect_config_count(ctypes.byref(c)))
    return c.value


def stencil_advect_config_select(ctx, index):
    return _check(lib().stencil_advect_config_select(ctx.handle, int(index)))


def stencil_residual(ctx, u, f, h, norms_dev, r=None, stream=None):
    """norms_dev: a float64 CUDA tensor of >= 2 elements (receives ||r||, ||f||)."""
    gu, gf = u.grid(), f.grid()
    gr = r.grid() if r is not None else None
    return _check(lib().stencil_residual(ctx.handle, ctypes.byref(gu), ctypes.byref(gf), float(h),
                                         ctypes.byref(gr) if gr is not None else None,
                                         ctypes.c_void_p(norms_dev.data_ptr()), _stream(stream)))


def stencil_residual_noalloc(u, f, h, norms_dev, r=None, stream=None):
    """stencil_residual without a context or any allocation (see
    include/stencil.h for its limit and the shared scratch it uses)."""
    gu, gf = u.grid(), f.grid()
    gr = r.grid() if r is not None else None
    return _check(lib().stencil_residual_noalloc(ctypes.byref(gu), ctypes.byref(gf), float(h),
                                                 ctypes.byref(gr) if gr is not None else None,
                                                 ctypes.c_void_p(norms_dev.data_ptr()), _stream(stream)))


def stencil_advect_uvw(ctx, u, v, w, su, sv, sw, tzc1, tzc2, tcx, tcy, stream=None):
    """tzc1, tzc2: float64 CUDA tensors of nz elements."""
    gs = [x.grid() for x in (u, v, w, su, sv, sw)]
    return _check(lib().stencil_advect_uvw(ctx.handle, *[ctypes.byref(g) for g in gs],
                                           ctypes.c_void_p(tzc1.data_ptr()), ctypes.c_void_p(tzc2.data_ptr()),
                                           float(tcx), float(tcy), _stream(stream)))


def _problems(us, fs, hs):
    arr = (stencil_problem * len(us))()
    for i, (u, f, h) in enumerate(zip(us, fs, hs)):
        arr[i].u = u.grid()
        arr[i].f = f.grid()
        arr[i].h = float(h)
    return arr


def stencil_batch_workspace_size(us, fs, hs):
    arr = _problems(us, fs, hs)
    n = ctypes.c_size_t()
    _check(lib().stencil_batch_workspace_size(arr, len(us), ctypes.byref(n)))
    return n.value


def stencil_batch_solve(ctx, us, fs, hs, rtol, inner_dtype=F32, max_sweeps=0, sweeps_per_cycle=0,
                        sweeps_per_pass=0, stall_ratio=0.0, workspace=None, stream=None, smoother=0):
    """Solve the instances (F64 Fields us, fs; spacings hs) in place.
    workspace: a CUDA tensor of >= stencil_batch_workspace_size bytes (one is
    allocated if None).  Returns a list of dicts (sweeps, cycles, status,
    rel_residual, final_dtype)."""
    import torch
    arr = _problems(us, fs, hs)
    need = stencil_batch_workspace_size(us, fs, hs)
    if workspace is None:
        workspace = torch.empty(need, dtype=torch.uint8, device=us[0].storage.device)
    assert workspace.numel() * workspace.element_size() >= need
    opts = stencil_batch_opts(float(rtol), int(max_sweeps), int(inner_dtype), int(sweeps_per_cycle),
                              int(sweeps_per_pass), int(smoother), float(stall_ratio))
    res = (stencil_result * len(us))()
    _check(lib().stencil_batch_solve(ctx.handle, arr, len(us), ctypes.byref(opts),
                                     ctypes.c_void_p(workspace.data_ptr()), need, res, _stream(stream)))
    return [{"sweeps": r.sweeps, "cycles": r.cycles, "status": r.status, "rel_residual": r.rel_residual,
             "final_dtype": r.final_dtype} for r in res]


class WsNet:
    """Owns a wsnet (the warm-start network; see include/stencil.h)."""

    def __init__(self, levels, channels, n, seed=0, device=0):
        h = ctypes.c_void_p()
        ch = (ctypes.c_int32 * len(channels))(*channels)
        _check(lib().wsnet_create(int(device), int(levels), ch, int(n), int(seed), ctypes.byref(h)))
        self.handle, self.levels, self.channels, self.n = h, levels, list(channels), n
        c = ctypes.c_int64()
        _check(lib().wsnet_num_params(h, ctypes.byref(c)))
        self.num_params = c.value

    def get_params(self):
        out = np.empty(self.num_params, dtype=np.float32)
        _check(lib().wsnet_get_params(self.handle, ctypes.c_void_p(out.ctypes.data), self.num_params))
        return out

    def set_params(self, arr):
        arr = np.ascontiguousarray(arr, dtype=np.float32)
        assert arr.size == self.num_params
        _check(lib().wsnet_set_params(self.handle, ctypes.c_void_p(arr.ctypes.data), self.num_params))

    def close(self):
        if self.handle:
            lib().wsnet_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def wsnet_save(net, path):
    return _check(lib().wsnet_save(net.handle, os.fsencode(path)))


def wsnet_load(net, path):
    return _check(lib().wsnet_load(net.handle, os.fsencode(path)))


def wsnet_use_tcgen05(net, enable):
    return _check(lib().wsnet_use_tcgen05(net.handle, int(bool(enable))))


def wsnet_status(net, stream=None):
    return _check(lib().wsnet_status(net.handle, _stream(stream)))


def wsnet_infer(net, f, u, stream=None):
    gf, gu = f.grid(), u.grid()
    return _check(lib().wsnet_infer(net.handle, ctypes.byref(gf), ctypes.byref(gu), _stream(stream)))


def wsnet_train_step(net, fs, us, lr, stream=None):
    """One Adam step over the samples (lists of F64 Fields); returns the loss."""
    af = (stencil_grid * len(fs))(*[f.grid() for f in fs])
    au = (stencil_grid * len(us))(*[u.grid() for u in us])
    loss = ctypes.c_double()
    _check(lib().wsnet_train_step(net.handle, af, au, len(fs), float(lr), ctypes.byref(loss), _stream(stream)))
    return loss.value


def wsnet_loss_grad(net, x, t, y=None, want_grads=True, stream=None):
    """x, t, y: float32 CUDA tensors of n^3 values.  Returns (loss, grads)."""
    grads = np.empty(net.num_params, dtype=np.float32) if want_grads else None
    loss = ctypes.c_double()
    _check(lib().wsnet_loss_grad(net.handle, ctypes.c_void_p(x.data_ptr()), ctypes.c_void_p(t.data_ptr()),
                                 ctypes.c_void_p(y.data_ptr()) if y is not None else None,
                                 ctypes.c_void_p(grads.ctypes.data) if grads is not None else None,
                                 ctypes.byref(loss), _stream(stream)))
    return loss.value, grads
