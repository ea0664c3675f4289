"""FP64 CPU oracle of the spiking-pixel U-Net stage (Sec. III-C of Bando et al.,
BIBM 2023): a U-Net applied to 64x64 patches of the two summary images
(S_i, T_i) of a segment, whose per-patch outputs are merged into one
probability map per segment by a weighted average over sliding patches.

TEST INFRASTRUCTURE ONLY (tests and the benchmark's CPU legs); the product
never imports it.  Plain numpy in double precision.

The paper fixes the input (two 64x64 summary patches), the output (a 64x64
map of spiking probabilities), the U-Net diagram convention, the sliding
patches and the weighted-average merge; the layer sizes were in a figure that
is not available.  Readings taken here:

  * four 2x2 max-pool steps (64 -> 4 px), two 3x3 convolutions with zero
    padding 1 and ReLU per level, 16 channels at 64x64 doubling per level to
    256 at 4x4; decoder: 2x2 stride-2 up-convolution (no activation) halving
    the channels, concatenation [skip, up], two 3x3 convolutions + ReLU;
    output 1x1 convolution 16 -> 1 and a logistic sigmoid;
  * input channels: S_i and T_i, each standardised over the whole image,
    (x - mean) / (std + 1e-3) with the population standard deviation;
  * patches every 32 px along each axis, plus one flush with the far border
    (positions min(32 j, n - 64)); images need H, W >= 64;
  * merge weight w(u) w(v), w(u) = min(u + 1, 64 - u) (a tent, 1 at the patch
    border, 32 at its centre); p(x) = sum w p_patch / sum w.

Parameter layout (flat float32): for every 3x3 convolution and up-convolution
in network order the weights, then the bias; convolution weights [Cout][Cin]
[3][3], up-convolution weights [Cin][Cout][2][2] (out[co][2y+i][2x+j] +=
in[ci][y][x] w[ci][co][i][j]); last the output weights [16] and bias [1].
Network order: enc0a enc0b enc1a enc1b enc2a enc2b enc3a enc3b bot_a bot_b
up3 dec3a dec3b up2 dec2a dec2b up1 dec1a dec1b up0 dec0a dec0b out.

The GPU runs the 3x3 and up-convolutions on BF16 weights and BF16 stored
activations with FP32 accumulation; `forward(..., act_round=round_bf16)`
applies the same roundings at the same points (the inputs z, every layer
output) so that the GPU can be compared tightly, and without it the oracle is
the plain FP64 network on the same (BF16) weights.

Parity: each layer pinned to torch's CPU conv2d / max_pool2d /
conv_transpose2d in float64 (library routines); the merge pinned by exact
reconstruction of a known map; the whole network pinned to a torch.nn
composition and to its closed form for zero weights (tests/test_unet_oracle.py).
"""
from __future__ import annotations

import math

import numpy as np

from .cnn import round_bf16  # nearest bfloat16, ties to even (pinned to torch's cast)

PATCH = 64
STRIDE = 32
LEVELS = 4
CH = [16, 32, 64, 128, 256]
EPS = 1e-3


def architecture():
    """[(kind, cin, cout)] in parameter order; kind in {'conv', 'up', 'out'}."""
    a = [("conv", 2, CH[0]), ("conv", CH[0], CH[0])]
    for l in range(1, LEVELS + 1):
        a += [("conv", CH[l - 1], CH[l]), ("conv", CH[l], CH[l])]
    for l in range(LEVELS - 1, -1, -1):
        a += [("up", CH[l + 1], CH[l]), ("conv", 2 * CH[l], CH[l]), ("conv", CH[l], CH[l])]
    a.append(("out", CH[0], 1))
    return a


def _wshape(kind, ci, co):
    if kind == "conv":
        return (co, ci, 3, 3)
    if kind == "up":
        return (ci, co, 2, 2)
    return (co * ci,)


def param_count() -> int:
    return sum(int(np.prod(_wshape(k, ci, co))) + co for k, ci, co in architecture())


def unpack(p):
    p = np.asarray(p, np.float64)
    assert p.size == param_count()
    out, o = [], 0
    for k, ci, co in architecture():
        shp = _wshape(k, ci, co)
        n = int(np.prod(shp))
        w = p[o:o + n].reshape(shp)
        o += n
        b = p[o:o + co]
        o += co
        out.append((k, w, b))
    return out


def bf16_weights(p):
    """The parameters as the GPU holds them: 3x3 and up-convolution weights in
    BF16, biases and the output layer in FP32."""
    p = np.asarray(p, np.float32).astype(np.float64)
    q = p.copy()
    o = 0
    for k, ci, co in architecture():
        n = int(np.prod(_wshape(k, ci, co)))
        if k != "out":
            q[o:o + n] = round_bf16(p[o:o + n])
        o += n + co
    return q


# ---- layers (NCHW, float64) --------------------------------------------------------
def conv3(x, w, b):
    """3x3 cross-correlation, zero padding 1, stride 1, plus bias."""
    n, ci, H, W = x.shape
    xp = np.zeros((n, ci, H + 2, W + 2))
    xp[:, :, 1:-1, 1:-1] = x
    y = np.zeros((n, w.shape[0], H, W)) + b[None, :, None, None]
    for ky in range(3):
        for kx in range(3):
            y += np.einsum("oc,nchw->nohw", w[:, :, ky, kx], xp[:, :, ky:ky + H, kx:kx + W])
    return y


def maxpool2(x):
    n, c, H, W = x.shape
    return x.reshape(n, c, H // 2, 2, W // 2, 2).max(axis=(3, 5))


def upconv2(x, w, b):
    """2x2 stride-2 transposed convolution: out[co][2y+i][2x+j] = b[co] +
    sum_ci x[ci][y][x] w[ci][co][i][j]."""
    n, ci, H, W = x.shape
    co = w.shape[1]
    y = np.zeros((n, co, 2 * H, 2 * W))
    for i in range(2):
        for j in range(2):
            y[:, :, i::2, j::2] = np.einsum("cd,nchw->ndhw", w[:, :, i, j], x)
    return y + b[None, :, None, None]


def sigmoid(v):
    return 1.0 / (1.0 + np.exp(-v))


def forward(params, x, act_round=None):
    """x [n][2][64][64] standardised summary patches -> probabilities [n][64][64].
    act_round: applied to the input and to every stored activation (the GPU's
    BF16 storage), or None for plain FP64."""
    rnd = act_round if act_round is not None else (lambda v: v)
    layers = unpack(params)
    it = iter(layers)

    def conv_relu(a):
        _, w, b = next(it)
        return rnd(np.maximum(conv3(a, w, b), 0.0))

    a = rnd(np.asarray(x, np.float64))
    skips = []
    for l in range(LEVELS + 1):
        if l > 0:
            a = maxpool2(a)
        a = conv_relu(conv_relu(a))
        skips.append(a)
    for l in range(LEVELS - 1, -1, -1):
        _, w, b = next(it)
        u = rnd(upconv2(a, w, b))
        a = np.concatenate([skips[l], u], axis=1)
        a = conv_relu(conv_relu(a))
    _, w, b = next(it)
    return sigmoid(np.einsum("c,nchw->nhw", w, a) + b[0])


# ---- patches and merge ---------------------------------------------------------------
def standardise(img):
    img = np.asarray(img, np.float64)
    m = img.mean()
    sd = math.sqrt(((img - m) ** 2).mean())
    return (img - m) / (sd + EPS)


def positions(n: int):
    """Patch origins along an axis of n >= 64 pixels."""
    assert n >= PATCH
    k = -(-(n - PATCH) // STRIDE) + 1
    return [min(STRIDE * j, n - PATCH) for j in range(k)]


def tent():
    u = np.arange(PATCH)
    w = np.minimum(u + 1, PATCH - u).astype(np.float64)
    return np.outer(w, w)


def patches(S, T):
    """Standardised (S, T) -> x [n_patches][2][64][64], patches row-major over
    (y positions, x positions)."""
    zs, zt = standardise(S), standardise(T)
    H, W = zs.shape
    out = []
    for y in positions(H):
        for x in positions(W):
            out.append(np.stack([zs[y:y + PATCH, x:x + PATCH], zt[y:y + PATCH, x:x + PATCH]]))
    return np.asarray(out)


def merge(probs, H, W):
    """Weighted average of per-patch maps [n_patches][64][64] (order of patches())."""
    acc = np.zeros((H, W))
    wsum = np.zeros((H, W))
    wt = tent()
    i = 0
    for y in positions(H):
        for x in positions(W):
            acc[y:y + PATCH, x:x + PATCH] += wt * probs[i]
            wsum[y:y + PATCH, x:x + PATCH] += wt
            i += 1
    return acc / wsum


def probability_maps(params, summary, act_round=None):
    """summary [k][2][H][W] (S_i, T_i) -> spiking-probability maps [k][H][W]."""
    summary = np.asarray(summary, np.float64)
    k, _, H, W = summary.shape
    q = bf16_weights(params)
    out = np.zeros((k, H, W))
    for i in range(k):
        x = patches(summary[i, 0], summary[i, 1])
        out[i] = merge(forward(q, x, act_round), H, W)
    return out
