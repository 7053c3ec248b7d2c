"""Pins for the mixed-precision refinement oracle.

Restarting the correction solve from e = 0 each cycle is exact: m sweeps of
A e = r from zero, added to u, equal m further sweeps of plain Jacobi on u.
So with an FP64 inner solve the refinement must reproduce plain Jacobi
iterates; with FP32/BF16 inner storage it must still reach the FP64 residual
target, checked by the oracle's own residual and by the DST solution."""
import numpy as np

import oracle
from oracle import exact
from paper_2310_01882_b300 import inputs


def test_f64_inner_equals_plain_jacobi():
    n = 10
    f = inputs.grf(n, seed=21)
    h = 1.0 / (n + 1)
    res = oracle.refine(np.zeros_like(f), f, h, rtol=0.0, inner="f64", m=7, max_sweeps=63)
    assert res["sweeps"] == 63 and res["cycles"] == 9 and res["status"] == -7
    plain = oracle.jacobi(np.zeros_like(f), f, h, 63)
    assert np.max(np.abs(res["u"] - plain)) <= 1e-13 * np.max(np.abs(plain))
    nr, nf = oracle.residual(plain, f, h)
    assert abs(res["rel"] - nr / nf) <= 1e-12 * nr / nf


def test_f32_inner_reaches_target():
    n = 12
    f = inputs.grf(n, seed=22)
    h = 1.0 / (n + 1)
    res = oracle.refine(np.zeros_like(f), f, h, rtol=1e-8, inner="f32", m=50)
    assert res["status"] == 0
    nr, nf = oracle.residual(res["u"], f, h)
    assert nr / nf <= 1e-8 and abs(res["rel"] - nr / nf) <= 1e-12
    ud = exact.solve(f, h)
    assert np.max(np.abs(res["u"] - ud)) <= 1e-6 * np.max(np.abs(ud))
    # same number of sweeps as plain FP64 Jacobi, to within one cycle
    plain_sweeps = 0
    u = np.zeros_like(f)
    while True:
        r, ff = oracle.residual(u, f, h)
        if r / ff <= 1e-8:
            break
        u = oracle.jacobi(u, f, h, 50)
        plain_sweeps += 50
    assert abs(res["sweeps"] - plain_sweeps) <= 50
    assert np.all(np.diff(res["hist"]) < 0)


def test_bf16_inner_converges():
    """BF16 inner storage still converges at the plain-Jacobi rate per cycle
    at this size (each cycle restarts e from zero)."""
    n = 24
    f = inputs.grf(n, seed=23)
    h = 1.0 / (n + 1)
    res = oracle.refine(np.zeros_like(f), f, h, rtol=1e-8, inner="bf16", m=100)
    nr, nf = oracle.residual(res["u"], f, h)
    assert nr / nf <= 1e-8
    assert res["final_inner"] == "bf16"
    mu = np.cos(np.pi / (n + 1))
    rates = res["hist"][2:] / res["hist"][1:-1]
    assert np.max(rates) <= 1.2 * mu ** 100


def test_stall_escalates_then_stops():
    """A cycle that reduces rel by less than stall_ratio escalates BF16 storage
    to FP32; a further stall in FP32 stops the solve (status -7), at a
    residual no worse than the last one evaluated."""
    n = 16
    f = inputs.grf(n, seed=25)
    h = 1.0 / (n + 1)
    res = oracle.refine(np.zeros_like(f), f, h, rtol=1e-8, inner="bf16", m=20, stall_ratio=0.2)
    assert res["final_inner"] == "f32" and res["status"] == -7
    hist = res["hist"]
    # the first stall is where the reduction fell short of 0.2
    k = next(i for i in range(1, len(hist)) if hist[i] > 0.2 * hist[i - 1])
    assert len(hist) > k + 1
    nr, nf = oracle.residual(res["u"], f, h)
    assert abs(nr / nf - res["rel"]) <= 1e-12 * res["rel"]


def test_nonfinite_source_reported():
    n = 6
    f = inputs.grf(n, seed=24)
    f[3, 3, 3] = np.nan
    res = oracle.refine(np.zeros_like(f), f, 1.0 / 7, rtol=1e-8)
    assert res["status"] == -6 and res["sweeps"] == 0


def test_redblack_f64_inner_equals_plain_redblack():
    """The same restart argument holds for any stationary linear iteration,
    so red-black inner sweeps with FP64 storage reproduce plain red-black
    Gauss-Seidel iterates."""
    n = 10
    f = inputs.grf(n, seed=24)
    h = 1.0 / (n + 1)
    res = oracle.refine(np.zeros_like(f), f, h, rtol=0.0, inner="f64", m=5, max_sweeps=40, smoother="redblack")
    assert res["sweeps"] == 40 and res["cycles"] == 8 and res["status"] == -7
    plain = oracle.rbgs(np.zeros_like(f), f, h, 40)
    assert np.max(np.abs(res["u"] - plain)) <= 1e-13 * np.max(np.abs(plain))


def test_redblack_f32_inner_reaches_target_in_about_half_the_sweeps():
    n = 12
    f = inputs.grf(n, seed=25)
    h = 1.0 / (n + 1)
    jac = oracle.refine(np.zeros_like(f), f, h, rtol=1e-8, inner="f32", m=20)
    rb = oracle.refine(np.zeros_like(f), f, h, rtol=1e-8, inner="f32", m=20, smoother="redblack")
    assert rb["status"] == 0 and jac["status"] == 0
    nr, nf = oracle.residual(rb["u"], f, h)
    assert nr / nf <= 1e-8
    # the asymptotic rate of red-black is the square of Jacobi's
    assert 0.4 * jac["sweeps"] <= rb["sweeps"] <= 0.6 * jac["sweeps"], (rb["sweeps"], jac["sweeps"])
