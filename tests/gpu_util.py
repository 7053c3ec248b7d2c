"""Helpers shared by the GPU parity tests (marshalling only)."""
import numpy as np

from paper_2310_01882_b300 import stencil as S


def rel_err(got, ref):
    """Normwise relative error max|got - ref| / max|ref| over the interior."""
    g = got[1:-1, 1:-1, 1:-1]
    r = ref[1:-1, 1:-1, 1:-1]
    den = np.max(np.abs(r))
    return float(np.max(np.abs(g - r)) / (den if den > 0 else 1.0))


def halo_equal(a, b):
    m = np.ones(a.shape, dtype=bool)
    m[1:-1, 1:-1, 1:-1] = False
    return np.array_equal(a[m], b[m])


_CTX = None


def ctx():
    global _CTX
    if _CTX is None:
        _CTX = S.Context(0)
    return _CTX


def sweep(u_np, f_np, h, nsweeps, dtype=S.F64, flags=S.SWEEP_AUTO, spp=0, work=True):
    """Run nsweeps through the C ABI; work=True passes an F64 workspace grid
    (the resident fixed-point path for F64), False passes NULL."""
    import torch
    u = S.Field.from_numpy(u_np, dtype)
    f = S.Field.from_numpy(f_np, dtype)
    t = u.like()
    w = S.Field(u.nx, u.ny, u.nz, S.F64) if work else None
    S.stencil_jacobi_sweep(ctx(), u, t, f, w, h, nsweeps, spp, flags)
    torch.cuda.synchronize()
    S.stencil_ctx_status(ctx())
    return u.to_numpy()
