"""Pins for the warm-start network oracle (oracle/net.py): the convolution
against a delta kernel, scipy's correlate and a brute-force voxel; adjoint
identities of every linear step; and the whole network's analytic gradient
against central finite differences."""
import numpy as np
import pytest
from scipy import ndimage

from oracle import net


def test_delta_kernel_is_identity():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((5, 6, 7, 3))
    W = np.zeros((3, 3, 3, 3, 3))
    W[1, 1, 1] = np.eye(3)
    b = np.array([0.5, -1.0, 2.0])
    assert np.array_equal(net.conv3(x, W, b), x + b)


def test_single_channel_matches_scipy_correlate():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((6, 5, 7))
    w = rng.standard_normal((3, 3, 3))
    ref = ndimage.correlate(x, w, mode="constant", cval=0.0)
    got = net.conv3(x[..., None], w[..., None, None], np.zeros(1))[..., 0]
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_brute_force_voxel():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((4, 4, 4, 2))
    W = rng.standard_normal((3, 3, 3, 2, 3))
    b = rng.standard_normal(3)
    out = net.conv3(x, W, b)
    for (z, y, xx) in [(0, 0, 0), (1, 2, 3), (3, 3, 3), (2, 0, 1)]:
        acc = b.copy()
        for dz in range(3):
            for dy in range(3):
                for dx in range(3):
                    zz, yy, xi = z + dz - 1, y + dy - 1, xx + dx - 1
                    if 0 <= zz < 4 and 0 <= yy < 4 and 0 <= xi < 4:
                        for ci in range(2):
                            for co in range(3):
                                acc[co] += x[zz, yy, xi, ci] * W[dz, dy, dx, ci, co]
        np.testing.assert_allclose(out[z, y, xx], acc, rtol=1e-12)


def test_adjoint_identities():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((4, 6, 8, 3))
    y = rng.standard_normal((2, 3, 4, 3))
    assert abs(np.sum(net.pool2(x) * y) - np.sum(x * net.pool2_bwd(y))) <= 1e-12
    z = rng.standard_normal((8, 12, 16, 3))
    assert abs(np.sum(net.up2(x) * z) - np.sum(x * net.up2_bwd(z))) <= 1e-11
    a = rng.standard_normal((5, 6, 7, 1))
    b = rng.standard_normal((5, 6, 7, 1))
    assert abs(np.sum(net.smooth121(a) * b) - np.sum(a * net.smooth121(b))) <= 1e-12
    W = rng.standard_normal((3, 3, 3, 3, 5))
    g = rng.standard_normal((4, 6, 8, 5))
    out = net.conv3(x, W, np.zeros(5))
    dx, dW, db = net.conv3_bwd(x, W, g)
    ip = np.sum(out * g)
    assert abs(ip - np.sum(x * dx)) <= 1e-10 * abs(ip)
    assert abs(ip - np.sum(W * dW)) <= 1e-10 * abs(ip)
    np.testing.assert_allclose(db, g.sum(axis=(0, 1, 2)))


def test_smoothing_filter_modes():
    """On sine modes sin(pi k i/(n+1)) (zero outside) the [1,2,1]/4 filter is
    diagonal with factor cos^2(pi k/(2(n+1))) per axis: the checkerboard
    mode k = n is multiplied by cos^2(pi n/(2(n+1))) ~ 1e-2 per axis and
    the smoothest mode by nearly 1."""
    n = 12
    i = np.arange(1, n + 1)
    for k in (1, 5, n):
        s = np.sin(np.pi * k * i / (n + 1))
        mode = s[:, None, None] * s[None, :, None] * s[None, None, :]
        fac = np.cos(np.pi * k / (2 * (n + 1))) ** 6
        np.testing.assert_allclose(net.smooth121(mode[..., None])[..., 0], fac * mode, atol=1e-14)


@pytest.mark.parametrize("channels", [[4, 6], [3, 4, 5]])
def test_network_gradient_finite_differences(channels):
    rng = np.random.default_rng(4)
    n = 8
    x = rng.standard_normal((n, n, n, 1))
    t = rng.standard_normal((n, n, n, 1)) * 0.1
    p = net.init_params(channels, seed=5)
    for k in p:
        if k.endswith(".b"):
            p[k] = rng.standard_normal(p[k].shape) * 0.1
    loss, grads, _ = net.loss_and_grads(p, x, t, channels)
    eps = 1e-6
    checked = 0
    for name in p:
        flat = p[name].reshape(-1)
        for idx in rng.choice(flat.size, size=min(3, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + eps
            lp = net.loss_and_grads(p, x, t, channels)[0]
            flat[idx] = old - eps
            lm = net.loss_and_grads(p, x, t, channels)[0]
            flat[idx] = old
            fd = (lp - lm) / (2 * eps)
            an = grads[name].reshape(-1)[idx]
            assert abs(fd - an) <= 1e-5 * max(abs(fd), 1e-4), (name, idx, fd, an)
            checked += 1
    assert checked >= 20


# ---- Adam (the optimiser of the warm-start training) -----------------------

def test_adam_first_step_closed_form():
    """From zero moments the bias corrections make m_hat = g and
    v_hat = g^2 exactly, so the first step moves each parameter by
    lr * g / (|g| + eps): about lr in the gradient's sign, and visibly less
    for a gradient near eps (1e-8 here: half of lr)."""
    g = np.array([0.3, -2.0, 1e-8, -1e-3, 0.0])
    p0 = np.array([1.0, -1.0, 0.5, 0.25, 2.0])
    p1, m1, v1 = net.adam_step(p0, g, np.zeros(5), np.zeros(5), 1, lr=0.01)
    want = p0 - 0.01 * g / (np.abs(g) + 1e-8)
    np.testing.assert_allclose(p1, want, rtol=1e-14, atol=1e-17)
    assert abs((p0[2] - p1[2]) - 0.005) <= 1e-12          # g = eps: half a step
    np.testing.assert_allclose(m1, 0.1 * g, rtol=1e-15)
    np.testing.assert_allclose(v1, 0.001 * g * g, rtol=1e-14)


def test_adam_constant_gradient_moves_lr_per_step():
    """With a constant gradient, m_t / c1 = g and v_t / c2 = g^2 for every
    t: each step moves by lr * g / (|g| + eps)."""
    g = np.array([0.7, -0.05])
    p = np.array([0.0, 0.0])
    m = v = np.zeros(2)
    for t in range(1, 6):
        p, m, v = net.adam_step(p, g, m, v, t, lr=0.1)
    np.testing.assert_allclose(p, -5 * 0.1 * g / (np.abs(g) + 1e-8), rtol=1e-12)


def test_adam_alternating_gradient_second_step():
    """g then -g: m_2 / c1 = -(1 - b1) / (1 + b1) g and v_2 / c2 = g^2,
    so the second step moves back by lr (1 - b1)/(1 + b1) g / (|g| + eps)."""
    g = np.array([0.2, -3.0])
    p1, m1, v1 = net.adam_step(np.zeros(2), g, np.zeros(2), np.zeros(2), 1, lr=0.05)
    p2, _, _ = net.adam_step(p1, -g, m1, v1, 2, lr=0.05)
    step2 = 0.05 * (0.1 / 1.9) * g / (np.abs(g) + 1e-8)
    np.testing.assert_allclose(p2 - p1, step2, rtol=1e-12)
