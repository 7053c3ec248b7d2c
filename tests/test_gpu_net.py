"""GPU parity of the warm-start network kernels (BF16 tensor-core 3x3x3
convolutions, pooling, upsampling, ReLU, output layer, loss and gradients)
against the FP64 network oracle run on the same bf16-rounded weights and
inputs with bf16 rounding of every stored activation."""
import numpy as np
import pytest

import oracle
from oracle import net as onet
from paper_2310_01882_b300 import inputs
from paper_2310_01882_b300 import stencil as S

pytestmark = pytest.mark.gpu


def bf16(a):
    return oracle.from_bf16(oracle.to_bf16(np.asarray(a, dtype=np.float32))).astype(np.float64)


def to_oracle_params(flat, channels, round_weights=True):
    """Device parameter vector -> oracle dict (weights (3,3,3,cin,cout))."""
    L = len(channels)
    p = {}
    off = 0
    names = onet.layer_names(L)
    dims = []
    for l in range(L):
        dims += [(1 if l == 0 else channels[l - 1], channels[l]), (channels[l], channels[l])]
    for l in range(L - 2, -1, -1):
        dims += [(channels[l + 1], channels[l]), (channels[l], channels[l])]
    for name, (ci, co) in zip(names, dims):
        w = flat[off:off + co * 27 * ci].astype(np.float64).reshape(co, 27, ci)
        off += co * 27 * ci
        w = w.transpose(1, 2, 0).reshape(3, 3, 3, ci, co)
        p[name + ".w"] = bf16(w) if round_weights else w
        p[name + ".b"] = flat[off:off + co].astype(np.float64)
        off += co
    p["out.w"] = flat[off:off + channels[0]].astype(np.float64).reshape(channels[0], 1)
    off += channels[0]
    p["out.b"] = flat[off:off + 1].astype(np.float64)
    off += 1
    assert off == flat.size
    return p, names, dims


def from_oracle_grads(g, channels):
    L = len(channels)
    parts = []
    for name in onet.layer_names(L):
        w = g[name + ".w"]
        ci, co = w.shape[3], w.shape[4]
        parts.append(w.reshape(27, ci, co).transpose(2, 0, 1).reshape(-1))
        parts.append(g[name + ".b"])
    parts.append(g["out.w"].reshape(-1))
    parts.append(g["out.b"].reshape(-1))
    return np.concatenate(parts)


@pytest.mark.parametrize("levels,channels,n,tc", [(2, [16, 32], 16, 1), (3, [16, 32, 64], 16, 1),
                                                   (3, [16, 32, 64], 32, 1), (3, [16, 32, 64], 32, 0),
                                                   (2, [16, 32], 128, 1)])
def test_forward_backward_match_oracle(levels, channels, n, tc):
    """tc = 1: the tcgen05 convolutions run wherever they apply (rows of 16
    to 128 voxels: levels 0 and 1 at n = 32; at n = 128 level 0 runs the
    row-halo kernel of the production 128^3 net, forward and input
    gradient); tc = 0: mma.sync everywhere."""
    import torch
    net = S.WsNet(levels, channels, n, seed=3)
    S.wsnet_use_tcgen05(net, tc)
    flat = net.get_params()
    rng = np.random.default_rng(7)
    # nonzero biases so every bias path is exercised
    flat = flat.copy()
    p0, names, dims = to_oracle_params(flat, channels, round_weights=False)
    off = 0
    for (ci, co) in dims:
        off += co * 27 * ci
        flat[off:off + co] = rng.standard_normal(co).astype(np.float32) * 0.05
        off += co
    net.set_params(flat)
    p, _, _ = to_oracle_params(flat, channels)
    x = rng.standard_normal((n, n, n)).astype(np.float32)
    t = (rng.standard_normal((n, n, n)) * 0.3).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    td = torch.from_numpy(t).cuda()
    yd = torch.zeros(n ** 3, dtype=torch.float32, device="cuda")
    loss, grads = S.wsnet_loss_grad(net, xd, td, yd)
    y_ref, cache = onet.forward(p, bf16(x)[..., None], channels, act_round=bf16)
    l_ref, gy = onet.mse(y_ref, t.astype(np.float64)[..., None])
    y = yd.cpu().numpy().reshape(n, n, n)
    assert np.max(np.abs(y - y_ref[..., 0])) <= 1e-2 * np.max(np.abs(y_ref)), np.max(np.abs(y - y_ref[..., 0]))
    assert abs(loss - l_ref) <= 1e-2 * l_ref
    g_ref = from_oracle_grads(onet.backward(p, cache, gy, channels), channels)
    # per layer, normwise relative error of the gradient
    off = 0
    for name, (ci, co) in zip(names, dims):
        for part, size in (("w", co * 27 * ci), ("b", co)):
            a, b = grads[off:off + size], g_ref[off:off + size]
            err = np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-30)
            assert err <= 3e-2, (name, part, err)
            off += size
    a, b = grads[off:], g_ref[off:]
    assert np.max(np.abs(a - b)) / np.max(np.abs(b)) <= 3e-2
    S.wsnet_status(net)
    net.close()


@pytest.mark.parametrize("n", [32, 64, 128])
def test_tcgen05_matches_mma_sync(n):
    """The two convolution paths agree on the same net and data (both are
    bf16 products with FP32 sums; only the summation order differs)."""
    import torch
    ch = [16, 32, 64, 64]
    net = S.WsNet(4, ch, n, seed=11)
    rng = np.random.default_rng(12)
    x = torch.from_numpy(rng.standard_normal((n, n, n)).astype(np.float32)).cuda()
    t = torch.from_numpy((rng.standard_normal((n, n, n)) * 0.3).astype(np.float32)).cuda()
    out = []
    for tc in (0, 1):
        S.wsnet_use_tcgen05(net, tc)
        y = torch.zeros(n ** 3, dtype=torch.float32, device="cuda")
        loss, g = S.wsnet_loss_grad(net, x, t, y)
        S.wsnet_status(net)
        out.append((loss, g, y.cpu().numpy()))
    (l0, g0, y0), (l1, g1, y1) = out
    assert np.max(np.abs(y0 - y1)) <= 1e-2 * np.max(np.abs(y0))
    assert abs(l0 - l1) <= 1e-2 * l0
    assert np.max(np.abs(g0 - g1)) <= 3e-2 * np.max(np.abs(g0))
    net.close()


def test_infer_scaling_and_halo():
    """wsnet_infer writes y * rms(f) / (3 pi^2) on the interior, halo kept."""
    import torch
    n = 16
    net = S.WsNet(2, [16, 32], n, seed=4)
    f = inputs.grf(n, seed=9) * 3.0
    u0 = np.zeros_like(f)
    u0[0] = 5.0
    fd, ud = S.Field.from_numpy(f), S.Field.from_numpy(u0)
    S.wsnet_infer(net, fd, ud)
    torch.cuda.synchronize()
    got = ud.to_numpy()
    rms = np.sqrt(np.mean(f[1:-1, 1:-1, 1:-1] ** 2))
    p, _, _ = to_oracle_params(net.get_params(), [16, 32])
    x = bf16(f[1:-1, 1:-1, 1:-1] / rms)[..., None]
    y, _ = onet.forward(p, x, [16, 32], act_round=bf16)
    ref = y[..., 0] * rms / (3 * np.pi ** 2)
    assert np.max(np.abs(got[1:-1, 1:-1, 1:-1] - ref)) <= 1e-2 * np.max(np.abs(ref))
    assert np.all(got[0] == 5.0) and np.all(got[-1] == 0.0)
    net.close()


def test_training_reduces_loss():
    """Adam on 4 fixed (source, solution) pairs of 16^3: the loss falls."""
    from oracle import exact
    n = 16
    net = S.WsNet(2, [16, 32], n, seed=5)
    fs, us = [], []
    for q in range(4):
        f = inputs.grf(n, seed=300 + q)
        fs.append(S.Field.from_numpy(f))
        us.append(S.Field.from_numpy(exact.solve(f, 1.0 / (n + 1))))
    losses = [S.wsnet_train_step(net, fs, us, 2e-3) for _ in range(40)]
    assert losses[-1] < 0.3 * losses[0], losses[::8]
    net.close()


def test_save_load_roundtrip(tmp_path):
    """wsnet_save / wsnet_load restore the parameters bit for bit (and the
    inference with them); a net of another shape refuses the file."""
    import torch
    n = 16
    a = S.WsNet(2, [16, 32], n, seed=21)
    b = S.WsNet(2, [16, 32], n, seed=22)
    path = str(tmp_path / "net.bin")
    S.wsnet_save(a, path)
    S.wsnet_load(b, path)
    assert np.array_equal(a.get_params(), b.get_params())
    f = S.Field.from_numpy(inputs.grf(n, seed=4))
    ua, ub = S.Field(n, n, n), S.Field(n, n, n)
    S.wsnet_infer(a, f, ua)
    S.wsnet_infer(b, f, ub)
    torch.cuda.synchronize()
    assert np.array_equal(ua.to_numpy(), ub.to_numpy())
    c = S.WsNet(2, [16, 16], n, seed=23)
    before = c.get_params()
    with pytest.raises(S.StencilError):
        S.wsnet_load(c, path)
    assert np.array_equal(before, c.get_params())
    for net in (a, b, c):
        net.close()


def test_checkpoint_resumes_training_exactly(tmp_path):
    """A checkpoint holds the parameters and the Adam state (moments and
    step count): training k steps, saving, loading into a fresh net and
    training k more gives bit for bit the parameters of 2k uninterrupted
    steps; a parameters-only load (the older file kind) does not."""
    n = 16
    fs = [S.Field.from_numpy(inputs.grf(n, seed=60 + i)) for i in range(4)]
    us = [S.Field.from_numpy(0.01 * inputs.grf(n, seed=70 + i)) for i in range(4)]

    def steps(net, first, last):
        for s in range(first, last):
            S.wsnet_train_step(net, fs[2 * (s % 2):2 * (s % 2) + 2], us[2 * (s % 2):2 * (s % 2) + 2], 1e-3)

    ref = S.WsNet(2, [16, 32], n, seed=31)
    steps(ref, 0, 6)
    a = S.WsNet(2, [16, 32], n, seed=31)
    steps(a, 0, 3)
    path = str(tmp_path / "ckpt.bin")
    S.wsnet_save(a, path)
    b = S.WsNet(2, [16, 32], n, seed=99)
    S.wsnet_load(b, path)
    steps(b, 3, 6)
    assert np.array_equal(b.get_params(), ref.get_params())
    c = S.WsNet(2, [16, 32], n, seed=99)
    c.set_params(a.get_params())   # parameters only: the optimiser restarts
    steps(c, 3, 6)
    assert not np.array_equal(c.get_params(), ref.get_params())
    for net in (ref, a, b, c):
        net.close()


def _read_checkpoint(path):
    """wsnet_save's file: parameters, the Adam step count and both moments."""
    import struct
    with open(path, "rb") as fh:
        raw = fh.read()
    assert raw[:8] == b"WSNET02\x00"
    L = struct.unpack_from("<i", raw, 8)[0]
    off = 12 + 4 * L + 4
    cnt = struct.unpack_from("<q", raw, off)[0]
    off += 8
    p = np.frombuffer(raw, dtype="<f4", count=cnt, offset=off).astype(np.float64)
    off += 4 * cnt
    step = struct.unpack_from("<q", raw, off)[0]
    off += 8
    m = np.frombuffer(raw, dtype="<f4", count=cnt, offset=off).astype(np.float64)
    v = np.frombuffer(raw, dtype="<f4", count=cnt, offset=off + 4 * cnt).astype(np.float64)
    return p, step, m, v


def test_adam_update_matches_oracle(tmp_path):
    """Each of three training steps applies the oracle's Adam update
    (oracle.net.adam_step: bias corrections, eps outside the square root)
    to the step's gradient, with the kernel's binary32 hyperparameters
    (0.999 as binary32 makes 1 - b2 differ from 0.001 by 1.3e-5): with the
    state saved before and after the step, the gradient is
    g = (m_t - b1 m_(t-1)) / (1 - b1), and the oracle's (p, v) from
    (p, m, v)_(t-1) and g equal the kernel's to binary32 rounding."""
    n = 16
    lr = 1e-3
    net = S.WsNet(2, [16, 32], n, seed=41)
    fs = [S.Field.from_numpy(inputs.grf(n, seed=80 + i)) for i in range(4)]
    us = [S.Field.from_numpy(0.01 * inputs.grf(n, seed=90 + i)) for i in range(4)]
    path = str(tmp_path / "s.bin")
    S.wsnet_save(net, path)
    prev = _read_checkpoint(path)
    assert prev[1] == 0 and not prev[2].any() and not prev[3].any()
    for t in range(1, 4):
        S.wsnet_train_step(net, fs[t - 1:t + 1], us[t - 1:t + 1], lr)
        S.wsnet_save(net, path)
        p, step, m, v = _read_checkpoint(path)
        assert step == t
        b1, b2, eps = (float(np.float32(x)) for x in (0.9, 0.999, 1e-8))
        g = (m - b1 * prev[2]) / (1.0 - b1)
        p_ref, m_ref, v_ref = onet.adam_step(prev[0], g, prev[2], prev[3], t, float(np.float32(lr)), b1, b2, eps)
        assert np.max(np.abs(v - v_ref)) <= 1e-6 * np.max(np.abs(v_ref)), t
        assert np.all(np.abs(p - p_ref) <= 2e-7 * np.abs(p_ref) + 1e-5 * lr), (t, np.max(np.abs(p - p_ref)))
        assert np.max(np.abs(prev[0] - p)) > 0.5 * lr        # the step moved the parameters
        prev = (p, step, m, v)
    net.close()
