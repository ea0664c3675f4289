"""Pins of the FP64 U-Net oracle (Sec. III-C: U-Net on 64x64 patches of the
summary pair, sliding patches merged by a weighted average) against library
routines, closed forms and exact reconstructions."""
import math

import numpy as np
import torch
import torch.nn.functional as F

import oracle.unet as U
from paper_2403_16438_gb300 import synth

rng = np.random.default_rng(7)


def test_conv3_is_torch_conv2d_same_padding():
    x = rng.normal(size=(2, 5, 9, 7))
    w = rng.normal(size=(4, 5, 3, 3))
    b = rng.normal(size=4)
    ref = F.conv2d(torch.from_numpy(x), torch.from_numpy(w), torch.from_numpy(b), padding=1)
    assert np.allclose(U.conv3(x, w, b), ref.numpy(), rtol=1e-12, atol=1e-12)


def test_maxpool_is_torch_max_pool2d():
    x = rng.normal(size=(3, 4, 8, 6))
    assert np.array_equal(U.maxpool2(x), F.max_pool2d(torch.from_numpy(x), 2).numpy())


def test_upconv_is_torch_conv_transpose2d():
    x = rng.normal(size=(2, 6, 4, 5))
    w = rng.normal(size=(6, 3, 2, 2))
    b = rng.normal(size=3)
    ref = F.conv_transpose2d(torch.from_numpy(x), torch.from_numpy(w), torch.from_numpy(b),
                             stride=2)
    assert np.allclose(U.upconv2(x, w, b), ref.numpy(), rtol=1e-12, atol=1e-12)


def _torch_unet(params):
    """The same reading composed from torch.nn layers (float64)."""
    layers = U.unpack(params)
    mods = []
    for kind, w, b in layers:
        if kind == "conv":
            m = torch.nn.Conv2d(w.shape[1], w.shape[0], 3, padding=1)
        elif kind == "up":
            m = torch.nn.ConvTranspose2d(w.shape[0], w.shape[1], 2, stride=2)
        else:
            m = torch.nn.Conv2d(w.shape[0], 1, 1)
            w = w.reshape(1, -1, 1, 1)
        m = m.double()
        with torch.no_grad():
            m.weight.copy_(torch.from_numpy(np.ascontiguousarray(w)))
            m.bias.copy_(torch.from_numpy(np.ascontiguousarray(b)))
        mods.append(m)

    def run(x):
        it = iter(mods)
        a, skips = x, []
        for l in range(5):
            if l:
                a = torch.nn.MaxPool2d(2)(a)
            a = torch.relu(next(it)(a))
            a = torch.relu(next(it)(a))
            skips.append(a)
        for l in range(3, -1, -1):
            u = next(it)(a)
            a = torch.cat([skips[l], u], 1)
            a = torch.relu(next(it)(a))
            a = torch.relu(next(it)(a))
        return torch.sigmoid(next(it)(a))[:, 0]
    return mods, run


def test_param_count_and_forward_match_a_torch_nn_composition():
    p = synth.unet_params(U.architecture(), seed=3).numpy()
    mods, run = _torch_unet(p)
    assert U.param_count() == sum(t.numel() for m in mods for t in m.parameters())
    x = rng.normal(size=(2, 2, 64, 64))
    with torch.no_grad():
        ref = run(torch.from_numpy(x)).numpy()
    assert np.allclose(U.forward(p, x), ref, rtol=1e-10, atol=1e-12)


def test_zero_weights_give_the_sigmoid_of_the_output_bias():
    p = np.zeros(U.param_count())
    p[-1] = 0.75  # exact in float32, the parameters' storage type
    S = rng.normal(size=(100, 130)) * 50 + 2000
    T = rng.random((100, 130)) * 20
    out = U.probability_maps(p, np.stack([S, T])[None])
    assert np.allclose(out, 1.0 / (1.0 + math.exp(-0.75)), rtol=0, atol=1e-15)


def test_positions_cover_the_image():
    assert U.positions(64) == [0]
    assert U.positions(512) == list(range(0, 449, 32))
    assert U.positions(100) == [0, 32, 36]
    for n in (64, 65, 96, 100, 128, 200, 511):
        cov = np.zeros(n, int)
        for p in U.positions(n):
            cov[p:p + 64] += 1
        assert cov.min() >= 1 and U.positions(n)[-1] == n - 64


def test_merge_reconstructs_a_map_cut_into_patches():
    """Patch outputs that are crops of one map merge back to that map exactly,
    whatever the weights; H != W catches a transposed index."""
    for H, W in ((128, 160), (100, 64), (64, 64)):
        M = rng.random((H, W))
        crops = [M[y:y + 64, x:x + 64] for y in U.positions(H) for x in U.positions(W)]
        assert np.allclose(U.merge(np.asarray(crops), H, W), M, rtol=0, atol=1e-14)


def test_merge_weights_are_the_tent():
    w = U.tent()
    assert w.shape == (64, 64) and np.array_equal(w, w.T)
    assert w[0, 0] == 1 and w[31, 31] == 32 * 32 and w[32, 32] == 32 * 32 and w[0, 31] == 32
    # two half-overlapping patches: at the overlap, the weighted average of 0 and 1
    H, W = 64, 96
    probs = np.stack([np.zeros((64, 64)), np.ones((64, 64))])
    m = U.merge(probs, H, W)
    u = np.arange(32, 64)
    wa = np.minimum(u + 1, 64 - u)        # weight of the first patch at column u
    wb = np.minimum(u - 32 + 1, 64 - (u - 32))
    assert np.allclose(m[10, 32:64], wb / (wa + wb), rtol=0, atol=1e-15)


def test_standardise():
    img = rng.normal(size=(70, 80)) * 13 + 400
    z = U.standardise(img)
    sd = img.std()
    assert abs(z.mean()) < 1e-12
    assert np.isclose(z.std(), sd / (sd + U.EPS), rtol=1e-12)
    assert np.array_equal(U.standardise(np.full((64, 64), 5.0)), np.zeros((64, 64)))


def test_bf16_weights_round_only_the_convolutions():
    p = synth.unet_params(U.architecture(), seed=1).numpy()
    q = U.bf16_weights(p)
    n_out = 16 + 1
    assert np.array_equal(q[-n_out:], p[-n_out:].astype(np.float64))
    first = 16 * 2 * 9
    assert np.array_equal(q[:first], U.round_bf16(p[:first]))
    assert np.array_equal(q[first:first + 16], p[first:first + 16].astype(np.float64))


def test_activation_rounding_stays_close_to_fp64():
    """The BF16 storage of activations moves the probabilities by at most a few
    hundredths on random weights (the tolerance the GPU is held to against the
    plain FP64 network)."""
    p = synth.unet_params(U.architecture(), seed=2).numpy()
    s = synth.summary_pair(synth.tiny_config(), 1, seed=5).numpy()
    a = U.probability_maps(p, s)
    b = U.probability_maps(p, s, act_round=U.round_bf16)
    assert np.abs(a - b).max() < 0.05
    assert 0.0 < a.min() and a.max() < 1.0
