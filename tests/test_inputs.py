"""The seeded input generators follow their stated recipes (they hold no
stencil arithmetic; these checks document the workloads): the k^-3
Gaussian random field, the winds, the vertical factors and the batch sizes."""
import numpy as np
from scipy.fft import dstn

from paper_2310_01882_b300 import inputs


def test_grf_recipe():
    n = 40
    a = inputs.grf(n, seed=2)
    assert a.shape == (n + 2,) * 3
    # zero Dirichlet halo, unit RMS interior, deterministic per seed
    for sl in (np.s_[0], np.s_[-1], np.s_[:, 0], np.s_[:, -1], np.s_[:, :, 0], np.s_[:, :, -1]):
        assert np.all(a[sl] == 0.0)
    assert abs(np.sqrt(np.mean(a[1:-1, 1:-1, 1:-1] ** 2)) - 1.0) < 1e-12
    assert np.array_equal(a, inputs.grf(n, seed=2)) and not np.array_equal(a, inputs.grf(n, seed=3))
    # power spectrum |k|^-3: the sine coefficients scaled by |k|^(3/2) are
    # iid N(0, s^2), so their variance is flat across |k| shells
    c = dstn(a[1:-1, 1:-1, 1:-1], type=1, norm="ortho")
    k = np.arange(1, n + 1, dtype=float)
    kk = np.sqrt(k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2)
    white = c * kk ** 1.5
    shells = [(kk >= lo) & (kk < lo + 8) for lo in (4, 16, 32, 48)]
    var = [np.var(white[s]) for s in shells]
    assert max(var) / min(var) < 1.15


def test_winds_recipe():
    u, v, w = inputs.winds(48, 40, 12)
    for a in (u, v, w):
        # periodic in x and y: the halo repeats the opposite interior edge
        assert np.array_equal(a[:, :, 0], a[:, :, -2]) and np.array_equal(a[:, :, -1], a[:, :, 1])
        assert np.array_equal(a[:, 0, :], a[:, -2, :]) and np.array_equal(a[:, -1, :], a[:, 1, :])
        rms = np.sqrt(np.mean(a[1:-1, 1:-1, 1:-1] ** 2))
        assert 3.0 < rms < 12.0   # about 7 m/s: 8 terms of amplitude 10/sqrt(8) plus N(0, 0.1)
    assert not np.array_equal(u, v)


def test_tzc_and_batch_sizes():
    t = inputs.tzc(256, 7)
    assert t.shape == (256,) and t.min() >= 0.5 and t.max() < 1.5
    sizes = inputs.batch_sizes()
    assert len(sizes) == 256 and min(sizes) >= 32 and max(sizes) <= 192
    assert sizes == inputs.batch_sizes()
