"""Training of the learned shift proposal with the library's own CUDA kernels.

Every step of the network (input crops and normalisation, forward, loss,
backward, Adam) runs in libvimg's kernels through the C ABI; torch only holds
the device buffers and generates the synthetic training frames
(``synth.training_batch``: paper-scale content, 128x128 centre crops, uniform
shifts in +-12 px).
"""
from __future__ import annotations

import ctypes
import math
import time

import torch

from . import synth
from .vimg import OK, VimgError, lib


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _ck(rc, what):
    if rc != OK:
        raise VimgError(rc, what)


def param_count() -> int:
    return lib.vimg_cnn_param_count()


def init_params(seed: int = 0, device="cuda") -> torch.Tensor:
    """He-normal convolution weights, zero biases, small linear weights."""
    g = torch.Generator().manual_seed(seed)
    chunks = []
    for cin in [2, 32, 32, 32, 32, 32]:
        std = math.sqrt(2.0 / (cin * 9))
        chunks.append(torch.randn(32 * cin * 9, generator=g) * std)
        chunks.append(torch.zeros(32))
    chunks.append(torch.randn(2 * 32, generator=g) * 0.05)
    chunks.append(torch.zeros(2))
    p = torch.cat(chunks).to(device=device, dtype=torch.float32).contiguous()
    assert p.numel() == param_count()
    return p


class Trainer:
    """Buffers for one batch size; step() runs one Adam step on a batch."""

    def __init__(self, params: torch.Tensor, batch: int, stream=None):
        self.p = params
        self.n = batch
        dev = params.device
        ws = lib.vimg_cnn_workspace_floats(batch)
        self.ws = torch.zeros(ws, device=dev)
        self.dws = torch.zeros(ws, device=dev)
        self.pb = torch.zeros(param_count(), dtype=torch.bfloat16, device=dev)
        self.g = torch.zeros_like(params)
        self.m = torch.zeros_like(params)
        self.v = torch.zeros_like(params)
        self.out = torch.zeros((batch, 2), device=dev)
        self.dout = torch.zeros((batch, 2), device=dev)
        self.loss = torch.zeros(1, device=dev)
        self.t = 0
        self.stream = stream or torch.cuda.current_stream(dev)
        self.sp = ctypes.c_void_p(self.stream.cuda_stream)

    def forward(self, frames, templates, template_stride):
        n, H, W = frames.shape
        _ck(lib.vimg_cnn_prepare(_p(frames), n, H, W, _p(templates), template_stride, _p(self.ws),
                                 self.sp), "prepare")
        _ck(lib.vimg_cnn_pack_bf16(_p(self.p), _p(self.pb), self.sp), "pack")
        _ck(lib.vimg_cnn_forward(_p(self.p), _p(self.pb), _p(self.ws), n, _p(self.out), self.sp),
            "forward")
        return self.out[:n]

    def step(self, frames, templates, targets, lr):
        n, H, W = frames.shape
        self.forward(frames, templates, H * W)
        _ck(lib.vimg_cnn_loss(_p(self.out), _p(targets), n, _p(self.dout), _p(self.loss),
                              self.sp), "loss")
        self.g.zero_()
        _ck(lib.vimg_cnn_backward(_p(self.p), _p(self.pb), _p(self.ws), _p(self.dws), n,
                                  _p(self.dout), _p(self.g), self.sp), "backward")
        self.t += 1
        _ck(lib.vimg_cnn_adam(_p(self.p), _p(self.g), _p(self.m), _p(self.v), lr, 0.9, 0.999,
                              1e-8, self.t, self.sp), "adam")
        return self.loss


def train(total_frames: int = 200_000, epochs: float = 4.0, batch: int = 256, lr: float = 2e-3,
          seed: int = 4000, n_scenes: int = 400, device="cuda", log_every: int = 0, params=None,
          pool=None):
    """Trains on a pool of `total_frames` synthetic frames (paper-scale content,
    128x128 centre crops, uniform shifts in +-12 px) for `epochs` passes with
    random symmetry augmentation; returns (params, history)."""
    dev = torch.device(device)
    if pool is None:
        pool = synth.training_pool(total_frames, n_scenes, seed, dev)
    g = torch.Generator().manual_seed(seed + 1)
    p = init_params(seed, dev) if params is None else params
    tr = Trainer(p, batch)
    steps = max(1, int(epochs * pool[0].shape[0] / batch))
    hist = []
    t0 = time.time()
    for s in range(steps):
        frames, tmpl, shifts = synth.augmented_batch(pool, batch, g)
        lr_s = lr * 0.5 * (1 + math.cos(math.pi * s / steps)) + 1e-5
        loss = tr.step(frames, tmpl, shifts.to(dev), lr_s)
        if log_every and (s % log_every == 0 or s == steps - 1):
            hist.append((s, float(loss.item()), time.time() - t0))
    return p, hist


@torch.no_grad()
def evaluate(params: torch.Tensor, n: int = 512, seed: int = 9999, n_scenes: int = 8,
             device="cuda"):
    """Proposal error on held-out scenes: returns |pred - planted| px [n, 2]."""
    dev = torch.device(device)
    scenes = synth.training_scenes(n_scenes, seed, dev)
    g = torch.Generator().manual_seed(seed + 1)
    tr = Trainer(params, n)
    frames, tmpl, shifts = synth.training_batch(scenes, n, g, dev)
    out = tr.forward(frames, tmpl, 128 * 128) * 12.0  # held-out scenes
    torch.cuda.synchronize()
    return (out.cpu() - shifts).abs()
