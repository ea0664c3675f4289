"""Pins of the FP64 oracle of the learned shift-proposal network: the forward
convolution against torch's CPU conv2d (a library routine) and the analytic
backward against central finite differences."""
import numpy as np
import pytest
import torch

from oracle import cnn


def rand_params(seed):
    r = np.random.default_rng(seed)
    p = []
    for c in cnn.IN_C:
        p += [r.normal(0, np.sqrt(2.0 / (9 * c)), 32 * c * 9), r.normal(0, 0.05, 32)]
    p += [r.normal(0, 0.1, 64), r.normal(0, 0.1, 2)]
    return np.concatenate(p)


def test_param_count():
    assert cnn.param_count() == 46914 == rand_params(0).size


@pytest.mark.parametrize("s", [1, 2])
def test_conv_matches_torch(s):
    r = np.random.default_rng(1)
    x = r.normal(0, 1, (2, 3, 9, 10))
    w = r.normal(0, 1, (32, 3, 3, 3))
    b = r.normal(0, 1, 32)
    ref = torch.nn.functional.conv2d(torch.from_numpy(x), torch.from_numpy(w), torch.from_numpy(b),
                                     stride=s, padding=1).numpy()
    assert np.max(np.abs(cnn.conv(x, w, b, s) - ref)) < 1e-12


def test_prepare_normalises_crops():
    r = np.random.default_rng(2)
    f = r.integers(0, 4000, (2, 140, 150)).astype(np.uint16)
    t = r.normal(3000, 100, (140, 150))
    x = cnn.prepare(f, t)
    assert x.shape == (2, 2, 128, 128)
    assert np.max(np.abs(x.mean(axis=(2, 3)))) < 1e-9
    assert np.max(np.abs(x.std(axis=(2, 3)) - 1)) < 1e-3
    np.testing.assert_allclose(x[0, 0, 0, 0] * (f[0, 6:134, 11:139].std() + 1e-3)
                               + f[0, 6:134, 11:139].mean(), f[0, 6, 11], rtol=1e-9)


def test_backward_matches_finite_differences():
    r = np.random.default_rng(3)
    p = rand_params(4)
    x = r.normal(0, 1, (2, 2, 128, 128))
    tgt = r.uniform(-12, 12, (2, 2))
    out, cache = cnn.forward(p, x)
    loss, dout = cnn.mse(out, tgt)
    g = cnn.backward(p, cache, dout)
    assert g.shape == p.shape
    # probe a few parameters of every layer with central differences
    offs = np.cumsum([0] + [32 * c * 9 + 32 for c in cnn.IN_C])
    idx = [int(o + k) for o in offs[:-1] for k in (0, 17, 32 * 9 - 1)] + [
        int(offs[-1] + 3), int(offs[-1] + 64)]
    eps = 1e-5
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += eps
        pm[i] -= eps
        lp, _ = cnn.mse(cnn.forward(pp, x)[0], tgt)
        lm, _ = cnn.mse(cnn.forward(pm, x)[0], tgt)
        fd = (lp - lm) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-6 + 1e-5 * abs(fd), (i, fd, g[i])


def test_round_bf16():
    v = np.array([1.0, 1.00390625, 1.005859375, -3.14159, 0.0], np.float32)
    r = cnn.round_bf16(v)
    assert r[0] == 1.0 and r[1] == 1.0  # tie to even
    assert r[2] == 1.0078125
    assert abs(r[3] + 3.140625) < 1e-12
