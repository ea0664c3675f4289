"""FP64 CPU oracle of the learned shift-proposal network.

TEST INFRASTRUCTURE ONLY (tests and the benchmark's CPU legs); the product
never imports it.  Plain numpy in double precision, written from the network's
definition (the paper has no such network; it is the proposal stage this
library adds in front of the Sec. II correlation):

  input  [2][128][128]: centre crops of the frame and of the template, each
         normalised as (x - mean) / (std + 1e-3) over its own crop
  conv1  3x3, stride 2, zero padding 1, 2 -> 32 channels, ReLU
  conv2..conv5 the same with 32 -> 32 channels; conv6 stride 1
  global average pool over the 4x4 map, linear 32 -> 2 (shift / 12 px)
  loss   (1/n) sum_b sum_j (out - target / 12)^2

Parameter layout (flat): per convolution w [32][c_in][3][3] then b [32];
then the linear weights [2][32] and bias [2].

Parity: forward pinned to torch's CPU conv2d (a library routine), backward
pinned to central finite differences (tests/test_cnn_oracle.py).
"""
from __future__ import annotations

import numpy as np

C = 32
IN_C = [2, 32, 32, 32, 32, 32]
STRIDE = [2, 2, 2, 2, 2, 1]
CROP = 128
SHIFT_SCALE = 12.0


def param_count() -> int:
    return sum(C * c * 9 + C for c in IN_C) + 2 * C + 2


def unpack(p):
    p = np.asarray(p, np.float64)
    layers, o = [], 0
    for c in IN_C:
        w = p[o:o + C * c * 9].reshape(C, c, 3, 3)
        o += C * c * 9
        b = p[o:o + C]
        o += C
        layers.append((w, b))
    lw = p[o:o + 2 * C].reshape(2, C)
    lb = p[o + 2 * C:o + 2 * C + 2]
    return layers, lw, lb


def prepare(frames, template):
    """frames uint16 [n][H][W]; template [H][W] or [n][H][W] -> x [n][2][128][128]."""
    frames = np.asarray(frames)
    n, H, W = frames.shape
    y0, x0 = (H - CROP) // 2, (W - CROP) // 2
    t = np.asarray(template, np.float64)
    if t.ndim == 2:
        t = np.broadcast_to(t, (n, H, W))
    x = np.zeros((n, 2, CROP, CROP))
    for b in range(n):
        for ch, img in enumerate((frames[b].astype(np.float64), t[b])):
            c = img[y0:y0 + CROP, x0:x0 + CROP]
            m = c.mean()
            sd = np.sqrt(((c - m) ** 2).mean())
            x[b, ch] = (c - m) / (sd + 1e-3)
    return x


def conv(x, w, b, s):
    """3x3 convolution, zero padding 1, stride s (cross-correlation, as in the
    network definition)."""
    n, ci, H, W = x.shape
    Ho, Wo = (H - 1) // s + 1, (W - 1) // s + 1
    xp = np.zeros((n, ci, H + 2, W + 2))
    xp[:, :, 1:-1, 1:-1] = x
    y = np.zeros((n, w.shape[0], Ho, Wo)) + b[None, :, None, None]
    for ky in range(3):
        for kx in range(3):
            xs = xp[:, :, ky:ky + s * (Ho - 1) + 1:s, kx:kx + s * (Wo - 1) + 1:s]
            y += np.einsum("oc,nchw->nohw", w[:, :, ky, kx], xs)
    return y


def forward(params, x):
    layers, lw, lb = unpack(params)
    acts = [x]
    a = x
    for (w, b), s in zip(layers, STRIDE):
        a = np.maximum(conv(a, w, b, s), 0.0)
        acts.append(a)
    g = a.mean(axis=(2, 3))
    out = g @ lw.T + lb
    return out, (acts, g)


def mse(out, target):
    d = out - np.asarray(target, np.float64) / SHIFT_SCALE
    n = out.shape[0]
    return (d ** 2).sum() / n, 2.0 * d / n


def backward(params, cache, dout):
    layers, lw, lb = unpack(params)
    acts, g = cache
    grads_layers = []
    glw = dout.T @ g
    glb = dout.sum(axis=0)
    dg = dout @ lw
    a6 = acts[-1]
    d = np.repeat(np.repeat(dg[:, :, None, None], a6.shape[2], 2), a6.shape[3], 3) / (
        a6.shape[2] * a6.shape[3])
    for li in range(len(layers) - 1, -1, -1):
        w, b = layers[li]
        s = STRIDE[li]
        a_out, a_in = acts[li + 1], acts[li]
        d = d * (a_out > 0)
        n, ci, H, W = a_in.shape
        Ho, Wo = a_out.shape[2], a_out.shape[3]
        xp = np.zeros((n, ci, H + 2, W + 2))
        xp[:, :, 1:-1, 1:-1] = a_in
        gw = np.zeros_like(w)
        dxp = np.zeros_like(xp)
        for ky in range(3):
            for kx in range(3):
                sl = (slice(None), slice(None), slice(ky, ky + s * (Ho - 1) + 1, s),
                      slice(kx, kx + s * (Wo - 1) + 1, s))
                gw[:, :, ky, kx] = np.einsum("nohw,nchw->oc", d, xp[sl])
                dxp[sl] += np.einsum("oc,nohw->nchw", w[:, :, ky, kx], d)
        grads_layers.append((gw, d.sum(axis=(0, 2, 3))))
        d = dxp[:, :, 1:-1, 1:-1]
    flat = []
    for gw, gb in reversed(grads_layers):
        flat += [gw.ravel(), gb]
    flat += [glw.ravel(), glb]
    return np.concatenate(flat)


def round_bf16(p):
    """Round float values to the nearest bfloat16 (ties to even), as float64."""
    u = np.asarray(p, np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)
