"""FP64 oracle of the warm-start network -- TEST INFRASTRUCTURE ONLY.

The learned warm start is not in the paper; its architecture is a reading of
the configuration "3D conv encoder-decoder, 4 levels, 16-32-64-64 channels,
3x3x3 kernels":
  * a U-Net: per level two 3x3x3 convolutions (zero padding, stride 1), each
    followed by ReLU; 2x2x2 average pooling between encoder levels; nearest
    2x upsampling between decoder levels, whose first convolution adds the
    encoder feature of the same level before its ReLU; a final 1x1x1
    convolution to one channel, no activation, followed by a fixed low-pass
    filter: the separable [1, 2, 1]/4 average along each axis (zero outside),
    which scales the sine mode k of an axis with n points by
    cos^2(pi k / (2 (n + 1))) and so all but removes the checkerboard mode --
    the mode plain Jacobi damps as slowly as the smoothest one;
  * no normalisation layers.
Fields are channels-last arrays (D, H, W, C).  Weights of a 3x3x3 layer are
(3, 3, 3, Cin, Cout) plus a bias (Cout,); the output layer is (Cin, 1).

Every operation is the plain definition (a correlation written as 27 shifted
matrix products, a mean over 2x2x2 blocks, a repeat); the backward pass is
the analytic adjoint of each.  `act_round` applies a rounding (e.g. to
bfloat16) to every stored activation, to follow a low-precision device
implementation step by step.
"""
import numpy as np


def conv3(x, W, b):
    """out[z,y,x,:] = b + sum over taps (dz,dy,dx) in {0,1,2}^3 of
    x[z+dz-1, y+dy-1, x+dx-1, :] @ W[dz,dy,dx] (zero outside)."""
    D, H, Wd, _ = x.shape
    pad = np.pad(x, ((1, 1), (1, 1), (1, 1), (0, 0)))
    out = np.zeros((D, H, Wd, W.shape[-1]))
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                out += pad[dz:dz + D, dy:dy + H, dx:dx + Wd, :] @ W[dz, dy, dx]
    return out + b


def conv3_bwd(x, W, g):
    """Adjoint of conv3: (dx, dW, db) for the output gradient g."""
    D, H, Wd, _ = x.shape
    pad = np.pad(x, ((1, 1), (1, 1), (1, 1), (0, 0)))
    dpad = np.zeros_like(pad)
    dW = np.zeros_like(W)
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                dpad[dz:dz + D, dy:dy + H, dx:dx + Wd, :] += g @ W[dz, dy, dx].T
                dW[dz, dy, dx] = np.tensordot(pad[dz:dz + D, dy:dy + H, dx:dx + Wd, :], g,
                                              axes=([0, 1, 2], [0, 1, 2]))
    return dpad[1:-1, 1:-1, 1:-1, :], dW, g.sum(axis=(0, 1, 2))


def pool2(x):
    D, H, W, C = x.shape
    return x.reshape(D // 2, 2, H // 2, 2, W // 2, 2, C).mean(axis=(1, 3, 5))


def pool2_bwd(g):
    return np.repeat(np.repeat(np.repeat(g, 2, 0), 2, 1), 2, 2) / 8.0


def up2(x):
    return np.repeat(np.repeat(np.repeat(x, 2, 0), 2, 1), 2, 2)


def up2_bwd(g):
    D, H, W, C = g.shape
    return g.reshape(D // 2, 2, H // 2, 2, W // 2, 2, C).sum(axis=(1, 3, 5))


def smooth121(y):
    """Separable [1,2,1]/4 filter along each of the three axes, zero padding
    (the filter is symmetric, so it is also its own adjoint)."""
    for ax in range(3):
        pad = [(0, 0)] * y.ndim
        pad[ax] = (1, 1)
        p = np.pad(y, pad)
        n = y.shape[ax]
        sl = lambda a, b: tuple(slice(a, b) if d == ax else slice(None) for d in range(y.ndim))  # noqa: E731
        y = 0.25 * p[sl(0, n)] + 0.5 * p[sl(1, n + 1)] + 0.25 * p[sl(2, n + 2)]
    return y


def relu(x):
    return np.maximum(x, 0.0)


def init_params(channels, seed, cin=1):
    """He-normal weights, zero biases, for the U-Net with these per-level
    channels.  Returns a dict of float64 arrays."""
    rng = np.random.default_rng(seed)
    p = {}

    def layer(name, ci, co):
        p[name + ".w"] = rng.standard_normal((3, 3, 3, ci, co)) * np.sqrt(2.0 / (27 * ci))
        p[name + ".b"] = np.zeros(co)

    L = len(channels)
    for l in range(L):
        layer(f"enc{l}a", cin if l == 0 else channels[l - 1], channels[l])
        layer(f"enc{l}b", channels[l], channels[l])
    for l in range(L - 2, -1, -1):
        layer(f"dec{l}a", channels[l + 1], channels[l])
        layer(f"dec{l}b", channels[l], channels[l])
    p["out.w"] = rng.standard_normal((channels[0], 1)) * np.sqrt(1.0 / channels[0])
    p["out.b"] = np.zeros(1)
    return p


def layer_names(L):
    names = []
    for l in range(L):
        names += [f"enc{l}a", f"enc{l}b"]
    for l in range(L - 2, -1, -1):
        names += [f"dec{l}a", f"dec{l}b"]
    return names


def forward(p, x, channels, act_round=None):
    """Network output y (D, H, W, 1) and the cache the backward pass needs."""
    rd = act_round if act_round is not None else (lambda a: a)
    L = len(channels)
    cache = {"x": x}
    h = x
    skips = []
    for l in range(L):
        if l > 0:
            h = rd(pool2(h))
            cache[f"pool{l}"] = h
        a = rd(relu(conv3(h, p[f"enc{l}a.w"], p[f"enc{l}a.b"])))
        cache[f"enc{l}a.in"], cache[f"enc{l}a.out"] = h, a
        b = rd(relu(conv3(a, p[f"enc{l}b.w"], p[f"enc{l}b.b"])))
        cache[f"enc{l}b.in"], cache[f"enc{l}b.out"] = a, b
        h = b
        skips.append(b)
    for l in range(L - 2, -1, -1):
        u = rd(up2(h))
        a = rd(relu(conv3(u, p[f"dec{l}a.w"], p[f"dec{l}a.b"]) + skips[l]))
        cache[f"dec{l}a.in"], cache[f"dec{l}a.out"] = u, a
        b = rd(relu(conv3(a, p[f"dec{l}b.w"], p[f"dec{l}b.b"])))
        cache[f"dec{l}b.in"], cache[f"dec{l}b.out"] = a, b
        h = b
    y = smooth121(h @ p["out.w"] + p["out.b"])
    cache["out.in"] = h
    return y, cache


def mse(y, t):
    """Mean squared error over every voxel (the network sees the interior)."""
    d = y - t
    return float(np.mean(d * d)), 2.0 * d / d.size


def backward(p, cache, gy, channels):
    """Analytic gradients of every parameter given dLoss/dy."""
    L = len(channels)
    grads = {}
    gy = smooth121(gy)
    h = cache["out.in"]
    grads["out.w"] = np.tensordot(h, gy, axes=([0, 1, 2], [0, 1, 2]))
    grads["out.b"] = gy.sum(axis=(0, 1, 2))
    g = gy @ p["out.w"].T
    gskip = [None] * L
    for l in range(0, L - 1):
        # decoder level l, in forward order l = L-2 .. 0; backward runs l = 0 .. L-2
        b_out = cache[f"dec{l}b.out"]
        g = g * (b_out > 0)
        g, grads[f"dec{l}b.w"], grads[f"dec{l}b.b"] = conv3_bwd(cache[f"dec{l}b.in"], p[f"dec{l}b.w"], g)
        a_out = cache[f"dec{l}a.out"]
        g = g * (a_out > 0)
        gskip[l] = g
        g, grads[f"dec{l}a.w"], grads[f"dec{l}a.b"] = conv3_bwd(cache[f"dec{l}a.in"], p[f"dec{l}a.w"], g)
        g = up2_bwd(g)
    for l in range(L - 1, -1, -1):
        if gskip[l] is not None:
            g = g + gskip[l]
        g = g * (cache[f"enc{l}b.out"] > 0)
        g, grads[f"enc{l}b.w"], grads[f"enc{l}b.b"] = conv3_bwd(cache[f"enc{l}b.in"], p[f"enc{l}b.w"], g)
        g = g * (cache[f"enc{l}a.out"] > 0)
        g, grads[f"enc{l}a.w"], grads[f"enc{l}a.b"] = conv3_bwd(cache[f"enc{l}a.in"], p[f"enc{l}a.w"], g)
        if l > 0:
            g = pool2_bwd(g)
    return grads


def loss_and_grads(p, x, t, channels):
    y, cache = forward(p, x, channels)
    loss, gy = mse(y, t)
    return loss, backward(p, cache, gy, channels), y


def adam_step(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba) of the parameters p with gradient g,
    first and second moments m, v, t the step number counted from 1, in
    binary64: m' = b1 m + (1 - b1) g, v' = b2 v + (1 - b2) g^2, bias
    corrections c1 = 1 - b1^t, c2 = 1 - b2^t, and
    p' = p - lr (m' / c1) / (sqrt(v' / c2) + eps).
    Returns (p', m', v')."""
    p, g, m, v = (np.asarray(a, dtype=np.float64) for a in (p, g, m, v))
    m1 = b1 * m + (1.0 - b1) * g
    v1 = b2 * v + (1.0 - b2) * g * g
    c1 = 1.0 - b1 ** t
    c2 = 1.0 - b2 ** t
    return p - lr * (m1 / c1) / (np.sqrt(v1 / c2) + eps), m1, v1
